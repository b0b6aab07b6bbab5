"""Plain FP64 oracle of the G-prox PDHG solve of one implicit reaction-diffusion step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests, smoke() and the
CPU-baseline leg of bench.py, never by the product library.

Everything is written for readability against the paper (arxiv 2305.03945):

  grid and Laplacians     Section 2.1 (periodic block-circulant Lap^P), Remark 1 (Neumann
                          Lap^N with the half-cell mirror ghost U_{-1} = U_0)
  residual map F          eq. (F(U) rd equation) for Allen-Cahn, eq. (F(U) CH) for
                          Cahn-Hilliard, Section 3.4.1 for the two-species Schnakenberg system
  adjoint Jacobian        the U-update of the G-prox dynamic (eqs. G-prox RD pdhg dynamic 3,
                          G-prox RD pdhg dynamic CH 3, Section 3.4.1 U/V updates)
  preconditioner          G = A_lin^2 (Section 2.1 "Choosing the matrix G"), or the
                          stabilised square of F's Jacobian with its nonlinear factor set to a
                          constant (Section 3.3's construction), inverted in the Fourier basis
                          (periodic) or DCT-II basis (Neumann), Section 2.1 "Application of
                          FFT" and Remark 1
  iteration               G-prox PDHG (eqs. G-prox linearized pdhg dynamic 1-3) inside
                          Algorithm 1, initial guess U_0 = U^k, P_0 = 0, extrapolation omega,
                          stopping rule ||Res(U_n)||_2 <= delta (Section 2.1 "Stopping criterion")

Conventions, and readings of the paper where it is silent or inconsistent:
  * arrays are ``[ncomp, ny, nx]``, x fastest; h_x = lx/nx, h_y = ly/ny for BOTH boundary
    conditions (Neumann nodes are cell centres, as in the paper's examples);
  * 3-D grids (nz > 1, arrays ``[ncomp, nz, ny, nx]``; not in the paper, which is 2-D): the same
    scheme with a third axis -- seven-point Laplacian, the symbol with a third sin^2 term, the
    transforms over all three axes;
  * Cahn-Hilliard: F(U) = (I + a dt Lap^2) U - U^k - b dt Lap W'(U), G = (I + a dt Lap^2)^2
    (the paper's lambda = -a sign reading of eq. (F(U) CH));
  * the stop test is applied to U_n before each update and ties go to "stop" (r <= delta);
  * a run is DIVERGED when the measure becomes non-finite or exceeds 1e8 times its first value;
    it is NOT_CONVERGED when ``max_iter`` updates did not reach the threshold.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

OK, NOT_CONVERGED, DIVERGED = "ok", "not_converged", "diverged"
DIVERGE_FACTOR = 1e8


# ----------------------------------------------------------------------------------------
# grid operators
# ----------------------------------------------------------------------------------------

def spacing(pb):
    """(h_x, h_y): side length over number of cells (Algorithm 1: h_x = L / N_x)."""
    return pb.lx / pb.nx, pb.ly / pb.ny


def spacing_z(pb):
    """h_z of a 3-D grid (the same rule along the third axis)."""
    return pb.lz / pb.nz


def _shift(u, axis, step, bc):
    """u at index i+step along ``axis`` with the boundary rule of ``bc``.

    periodic: wrap around (block-circulant Lap^P, Section 2.1);
    neumann : half-cell mirror ghost, U_{-1} = U_0 and U_N = U_{N-1} (Remark 1).
    """
    if bc == "periodic":
        return np.roll(u, -step, axis=axis)
    n = u.shape[axis]
    idx = np.arange(n) + step
    idx = np.where(idx < 0, -1 - idx, idx)
    idx = np.where(idx >= n, 2 * n - 1 - idx, idx)
    return np.take(u, idx, axis=axis)


def lap(u, pb):
    """Five-point Laplacian (x_{i,j+1} + x_{i,j-1} - 2x)/h_x^2 + (x_{i+1,j} + x_{i-1,j} - 2x)/h_y^2;
    on a 3-D grid the seven-point one, with (x_{l+1} + x_{l-1} - 2x)/h_z^2 along z added."""
    hx, hy = spacing(pb)
    out = ((_shift(u, -1, 1, pb.bc) + _shift(u, -1, -1, pb.bc) - 2 * u) / hx ** 2
           + (_shift(u, -2, 1, pb.bc) + _shift(u, -2, -1, pb.bc) - 2 * u) / hy ** 2)
    if pb.nz > 1:
        out = out + (_shift(u, -3, 1, pb.bc) + _shift(u, -3, -1, pb.bc) - 2 * u) / spacing_z(pb) ** 2
    return out


def symbol_mu(pb):
    """Nonnegative eigenvalues mu of -Lap on the transform grid, shape [ny, nx].

    periodic: mu = 4/h_x^2 sin^2(pi kx/nx) + 4/h_y^2 sin^2(pi ky/ny)   (Fourier modes)
    neumann : mu = 4/h_x^2 sin^2(pi kx/(2nx)) + 4/h_y^2 sin^2(pi ky/(2ny))   (DCT-II modes)
    """
    hx, hy = spacing(pb)
    kx = np.arange(pb.nx)[None, :]
    ky = np.arange(pb.ny)[:, None]
    d = 1.0 if pb.bc == "periodic" else 2.0
    mu = (4 / hx ** 2 * np.sin(np.pi * kx / (d * pb.nx)) ** 2
          + 4 / hy ** 2 * np.sin(np.pi * ky / (d * pb.ny)) ** 2)
    if pb.nz > 1:   # 3-D: shape [nz, ny, nx], a third sin^2 term along z
        kz = np.arange(pb.nz)[:, None, None]
        mu = mu[None] + 4 / spacing_z(pb) ** 2 * np.sin(np.pi * kz / (d * pb.nz)) ** 2
    return mu


# ----------------------------------------------------------------------------------------
# the implicit step: F, its adjoint Jacobian, the preconditioner symbol
# ----------------------------------------------------------------------------------------

def check_problem(pb):
    if pb.kind in ("allen_cahn", "gray_scott", "schnakenberg") and pb.op != "laplacian":
        raise ValueError("%s needs op='laplacian'" % pb.kind)
    if pb.kind in ("ch_implicit", "ch_split") and pb.op != "neg_biharmonic":
        raise ValueError("%s needs op='neg_biharmonic'" % pb.kind)
    if (pb.kind == "fch") != (pb.op == "functionalized"):
        raise ValueError("kind 'fch' goes with op='functionalized' and only with it")


# Sixth-order functionalized Cahn-Hilliard (Section 3.3, eq. 6thorder) with a = eps^2 and b
# scaling the double well W(u) = (u^2 - 1)^2 / 4:
#   mu(U) = a Lap U - b W'(U)                  (W' = u^3 - u)
#   A(U)  = a Lap - b diag(W''(U)) + a I       (W'' = 3u^2 - 1: the paper prints 3u^2, but its
#                                               own remark that W'' is about 2 at u = +-1 fixes
#                                               the minus one; W^(3) = 6u)
#   F(U)  = U - U^k - dt Lap A(U) mu(U)
def _fch_mu(pb, U):
    return pb.a * lap(U, pb) - pb.b * (U ** 3 - U)


def _fch_A(pb, U, x):
    return pb.a * lap(x, pb) - pb.b * (3 * U ** 2 - 1) * x + pb.a * x


def residual(pb, U, Uk):
    """F(U) whose root is the implicit step U^{k+1}; arrays [ncomp, ny, nx]."""
    dt, a, b = pb.dt, pb.a, pb.b
    L = lambda x: lap(x, pb)
    if pb.kind == "none":
        if pb.op == "laplacian":                      # (I - a dt Lap) U - U^k
            return U - Uk - dt * a * L(U)
        return U + dt * a * L(L(U)) - Uk              # (I + a dt Lap^2) U - U^k
    if pb.kind == "allen_cahn":                       # eq. (F(U) rd equation), f = -b W'
        f = -b * (U ** 3 - U)
        return U - Uk - dt * (a * L(U) + f)
    if pb.kind == "ch_implicit":                      # eq. (F(U) CH), sign reading lambda=-a
        return U + dt * a * L(L(U)) - Uk - dt * b * L(U ** 3 - U)
    if pb.kind == "ch_split":                         # convex part U^3 implicit, -U explicit
        return U + dt * a * L(L(U)) - Uk - dt * b * L(U ** 3) + dt * b * L(Uk)
    if pb.kind == "gray_scott":
        Du, Dv, Ff, k = pb.p
        u, v = U[0], U[1]
        Fu = u - Uk[0] - dt * (Du * L(u) - u * v * v + Ff * (1 - u))
        Fv = v - Uk[1] - dt * (Dv * L(v) + u * v * v - (Ff + k) * v)
        return np.stack([Fu, Fv])
    if pb.kind == "fch":                              # Section 3.3, F(U) of the 6th-order flow
        return U - Uk - dt * L(_fch_A(pb, U, _fch_mu(pb, U)))
    if pb.kind == "schnakenberg":                     # Section 3.4.1, F_u and F_v
        D1, D2, kap, a_s, b_s = pb.p
        u, v = U[0], U[1]
        Fu = u - Uk[0] - dt * (D1 * L(u) + kap * (a_s - u + u * u * v))
        Fv = v - Uk[1] - dt * (D2 * L(v) + kap * (b_s - u * u * v))
        return np.stack([Fu, Fv])
    raise ValueError(pb.kind)


def grad_F_T(pb, U, Pt):
    """nabla_U F(U)^T applied to the extrapolated dual Pt (the U-update of the dynamic)."""
    dt, a, b = pb.dt, pb.a, pb.b
    L = lambda x: lap(x, pb)
    if pb.kind == "none":
        if pb.op == "laplacian":
            return Pt - dt * a * L(Pt)
        return Pt + dt * a * L(L(Pt))
    if pb.kind == "allen_cahn":                       # eq. (G-prox RD pdhg dynamic 3)
        fprime = -b * (3 * U ** 2 - 1)
        return Pt - dt * a * L(Pt) - dt * fprime * Pt
    if pb.kind == "ch_implicit":                      # eq. (G-prox RD pdhg dynamic CH 3)
        return Pt + dt * a * L(L(Pt)) - dt * b * (3 * U ** 2 - 1) * L(Pt)
    if pb.kind == "ch_split":
        return Pt + dt * a * L(L(Pt)) - dt * b * (3 * U ** 2) * L(Pt)
    if pb.kind == "gray_scott":
        Du, Dv, Ff, k = pb.p
        u, v = U[0], U[1]
        P, Q = Pt[0], Pt[1]
        gu = P - dt * Du * L(P) + dt * (v * v + Ff) * P - dt * v * v * Q
        gv = Q - dt * Dv * L(Q) + 2 * dt * u * v * P - dt * (2 * u * v - (Ff + k)) * Q
        return np.stack([gu, gv])
    if pb.kind == "fch":
        # dF = I - dt Lap (A(U) B(U) - b diag(W^(3)(U) mu)) with B = a Lap - b diag(W''(U)), so
        # dF^T P = P - dt B A Lap P + dt b mu W^(3) Lap P (Lap, A and B are symmetric): the
        # U-update of Section 3.3
        q = L(Pt)
        r = _fch_A(pb, U, q)
        s = a * L(r) - b * (3 * U ** 2 - 1) * r
        return Pt - dt * s + dt * b * _fch_mu(pb, U) * (6 * U) * q
    if pb.kind == "schnakenberg":                     # Section 3.4.1 U_{n+1}, V_{n+1} updates
        D1, D2, kap, a_s, b_s = pb.p
        u, v = U[0], U[1]
        P, Q = Pt[0], Pt[1]
        gu = P - dt * (D1 * L(P) + kap * (-P + 2 * u * v * (P - Q)))
        gv = Q - dt * (D2 * L(Q) + kap * (u * u * (P - Q)))
        return np.stack([gu, gv])
    raise ValueError(pb.kind)


def ghat(pb):
    """Eigenvalues of the preconditioner G on the transform grid, shape [ncomp, ny, nx].

    G = A_lin^2 with A_lin the linear, constant-coefficient part of F:
      laplacian op      A_lin = I - D dt Lap    ->  g = (1 + D dt mu)^2   (D = a, or per species)
      neg_biharmonic    A_lin = I + a dt Lap^2  ->  g = (1 + a dt mu^2)^2
      functionalized    A_lin = I - dt Lap (a Lap - (2b - a) I) a Lap, W'' replaced by its value
                        2b at u = +-1 (Section 3.3)  ->  g = (1 + dt a mu^2 (a mu + 2b - a))^2
    precond 'none' gives G = I (plain linearised PDHG, eqs. illustrate pdhg dynamic 1-3).
    precond 'stabilized' squares the Jacobian of F with its nonlinear factor replaced by the
    constant s = pb.shift (Section 3.3's idea, for any scalar reaction): Allen-Cahn
    A = (1 + b dt s) I - a dt Lap; Cahn-Hilliard A = I + a dt Lap^2 - b s dt Lap (s in place of
    W''(U), or of 3 U^2 for the convex split); sixth-order A as above with (s b - a).
    """
    if pb.precond == "none":
        return np.ones(pb.shape)
    mu = symbol_mu(pb)
    dt = pb.dt
    if pb.precond == "stabilized":
        if pb.kind not in ("allen_cahn", "ch_implicit", "ch_split", "fch"):
            raise ValueError("the stabilized preconditioner needs a scalar reaction")
        s = pb.shift
        if pb.op == "laplacian":
            return ((1 + pb.b * dt * s + pb.a * dt * mu) ** 2)[None]
        if pb.op == "functionalized":
            return ((1 + dt * pb.a * mu ** 2 * (pb.a * mu + s * pb.b - pb.a)) ** 2)[None]
        return ((1 + pb.b * s * dt * mu + pb.a * dt * mu ** 2) ** 2)[None]
    if pb.kind in ("gray_scott", "schnakenberg"):
        d1, d2 = pb.p[0], pb.p[1]
        return np.stack([(1 + d1 * dt * mu) ** 2, (1 + d2 * dt * mu) ** 2])
    if pb.op == "laplacian":
        return ((1 + pb.a * dt * mu) ** 2)[None]
    if pb.op == "functionalized":
        return ((1 + dt * pb.a * mu ** 2 * (pb.a * mu + 2 * pb.b - pb.a)) ** 2)[None]
    return ((1 + pb.a * dt * mu ** 2) ** 2)[None]


def apply_ginv(pb, W, g=None):
    """Y = G^{-1} W: 2-D FFT (periodic) or orthonormal DCT-II / DCT-III (Neumann), divide by g."""
    if g is None:
        g = ghat(pb)
    if pb.precond == "none":
        return W.copy()
    ax = (-3, -2, -1) if pb.nz > 1 else (-2, -1)
    if pb.bc == "periodic":
        return np.real(np.fft.ifftn(np.fft.fftn(W, axes=ax) / g, axes=ax))
    Wh = sfft.dctn(W, type=2, axes=ax, norm="ortho")
    return sfft.idctn(Wh / g, type=2, axes=ax, norm="ortho")


def measure(pb, W, Uk):
    """(r, threshold) of the stopping rule; r sums the l2 norms of the components of F."""
    s = sum(np.sqrt(np.sum(W[c] * W[c])) for c in range(W.shape[0]))
    if pb.tol_kind == "res_abs":                      # ||Res||_2 = ||F||_2 / h_t <= delta
        return s / pb.dt, pb.tol
    return s, pb.tol * np.sqrt(np.sum(Uk * Uk))


# ----------------------------------------------------------------------------------------
# Algorithm 1: PDHG for one implicit step, then the time loop
# ----------------------------------------------------------------------------------------

def pdhg_step(pb, Uk, history=False, U0=None):
    """Solve F(U) = 0 for one implicit step from U^k by G-prox PDHG.

    Returns (U, info) with info = {iterations, status, residual, history}.  ``iterations``
    counts updates of (U, P); the returned U is the first iterate whose measure is <= the
    threshold (or the last one on NOT_CONVERGED / DIVERGED).
    """
    check_problem(pb)
    Uk = np.asarray(Uk, dtype=np.float64)
    U = Uk.copy() if U0 is None else np.array(U0, dtype=np.float64)
    P = np.zeros_like(U)
    g = ghat(pb)
    hist = []
    r0 = None
    n = 0
    while True:
        W = residual(pb, U, Uk)                       # W_n = F(U_n)
        r, thresh = measure(pb, W, Uk)
        hist.append(r)
        if r0 is None:
            r0 = r
        if r <= thresh:
            status = OK
            break
        if not np.isfinite(r) or r > DIVERGE_FACTOR * r0:
            status = DIVERGED
            break
        if n == pb.max_iter:
            status = NOT_CONVERGED
            break
        Y = apply_ginv(pb, W, g)                      # solve G Y = W
        Pt = P + (1 + pb.omega) * pb.tau_p * Y        # P~ = P_{n+1} + omega (P_{n+1} - P_n)
        P = P + pb.tau_p * Y                          # P_{n+1} = P_n + tau_p G^{-1} F(U_n)
        U = U - pb.tau_u * grad_F_T(pb, U, Pt)        # U_{n+1} = U_n - tau_u dF(U_n)^T P~
        n += 1
    info = {"iterations": n, "status": status, "residual": r}
    if history:
        info["history"] = np.array(hist)
    return U, info


def solve(pb, u0, nsteps, history=False):
    """Algorithm 1's outer loop: ``nsteps`` implicit steps from u0.  Returns (U, infos)."""
    U = np.array(u0, dtype=np.float64).reshape(pb.shape)
    infos = []
    for _ in range(nsteps):
        U, info = pdhg_step(pb, U, history=history)
        infos.append(info)
        if info["status"] != OK:
            break
    return U, infos


# ----------------------------------------------------------------------------------------
# diagnostics used by invariant tests
# ----------------------------------------------------------------------------------------

def mass(pb, U):
    hx, hy = spacing(pb)
    hz = spacing_z(pb) if pb.nz > 1 else 1.0
    return hx * hy * hz * float(np.sum(U))


def ac_energy(pb, U):
    """Discrete Allen-Cahn / Cahn-Hilliard energy (eq. AC, CH energy):
    h_x h_y sum [ a/2 |grad_h u|^2 + b (u^2-1)^2/4 ], with the forward differences over the
    edges of the grid graph of each boundary condition (periodic: wrap edges included;
    Neumann: interior edges only)."""
    hx, hy = spacing(pb)
    u = U[0]
    if pb.bc == "periodic":
        dx = (np.roll(u, -1, axis=1) - u) / hx
        dy = (np.roll(u, -1, axis=0) - u) / hy
    else:
        dx = np.diff(u, axis=1) / hx
        dy = np.diff(u, axis=0) / hy
    grad2 = np.sum(dx * dx) + np.sum(dy * dy)
    return hx * hy * (0.5 * pb.a * grad2 + pb.b * np.sum((u * u - 1) ** 2) / 4)
