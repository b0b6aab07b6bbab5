"""Seeded synthetic inputs and problem records for the implicit reaction-diffusion step.

This module holds parameter records and input generators only: it contains none of the
method's arithmetic (no stencil, residual, preconditioner or PDHG update). Both the CPU
oracle and the GPU path take their inputs from here and from nowhere else.

Every generator is deterministic in its seed (numpy PCG64).  The shapes, parameters and
initial-condition recipes follow the implicit-step workloads of the paper (Section 3) and
the five synthetic configurations built on them:

  * ``config_allen_cahn_periodic``   Allen-Cahn, 64x64, [0,2pi)^2, a=eps=0.1, b=1/eps, dt=0.01
  * ``config_allen_cahn_neumann``    Allen-Cahn, 1024x1024, [0,1]^2 cell-centred, eps=0.01
  * ``config_cahn_hilliard_split``   Cahn-Hilliard convex-concave split, 512x512, eps=0.02
  * ``config_gray_scott``            Gray-Scott 2048x2048x2, [0,2.5)^2
  * ``config_schnakenberg``          Schnakenberg (Section 3.4.1), 128x128 Neumann

Array layout: ``[ncomp, ny, nx]`` float64, x fastest (row-major), i.e. the vectorisation
``l = i*nx + j`` of the paper's Section 2.1 with i the y index and j the x index.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

# reaction kinds, boundary conditions, operators, preconditioners and stopping rules.
KINDS = ("none", "allen_cahn", "ch_implicit", "ch_split", "gray_scott", "schnakenberg", "fch")
TWO_SPECIES = ("gray_scott", "schnakenberg")
BCS = ("periodic", "neumann")
OPS = ("laplacian", "neg_biharmonic", "functionalized")
PRECONDS = ("none", "linear")
TOL_KINDS = ("res_abs", "f_rel")


@dataclass(frozen=True)
class Problem:
    """Parameters of one implicit time step solved by G-prox PDHG.

    kind            reaction term (see ``KINDS``)
    op              'laplacian' (L = a*Lap) or 'neg_biharmonic' (L = -a*Lap^2)
    a, b            diffusion and reaction scales (Allen-Cahn / Cahn-Hilliard, Section 3.1-3.2)
    p               kind-specific parameters:
                      gray_scott:   (Du, Dv, F, k)
                      schnakenberg: (D1, D2, kappa, a_s, b_s)
    dt              physical time step h_t
    tau_u, tau_p    PDHG primal / dual step sizes
    omega           extrapolation coefficient (1 in all of the paper's experiments)
    precond         'linear' (G = A_lin^2, Section 2.1 "Choosing the matrix G"), 'none', or
                    'stabilized' (A_lin with the nonlinear factor replaced by the constant `shift`,
                    the idea of Section 3.3)
    shift           the constant of the 'stabilized' preconditioner: in place of W''(U) for
                    Allen-Cahn, implicit Cahn-Hilliard and the sixth-order equation, of 3 U^2
                    for the convex split (2, resp. 3, at u = +-1)
    tol, tol_kind   'res_abs': stop when sum_c ||F_c(U)||_2 / dt <= tol   (Section 2.1 stopping rule)
                    'f_rel'  : stop when sum_c ||F_c(U)||_2 <= tol * ||U^k||_2
    max_iter        cap on PDHG iterations per time step
    nz, lz          points and side length along z of a 3-D grid (nz = 1: a 2-D grid); the
                    3-D problem is the paper's scheme with a third axis (7-point Laplacian,
                    separable 3-D transforms)
    """

    nx: int
    ny: int
    lx: float
    ly: float
    bc: str
    op: str
    kind: str
    dt: float
    a: float = 0.0
    b: float = 0.0
    p: tuple = ()
    tau_u: float = 0.8
    tau_p: float = 0.8
    omega: float = 1.0
    precond: str = "linear"
    shift: float = 0.0
    tol: float = 1e-10
    tol_kind: str = "res_abs"
    max_iter: int = 10000
    nz: int = 1
    lz: float = 1.0

    @property
    def ncomp(self) -> int:
        return 2 if self.kind in TWO_SPECIES else 1

    @property
    def ndim(self) -> int:
        return 3 if self.nz > 1 else 2

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> tuple:
        """[ncomp, ny, nx] on 2-D grids, [ncomp, nz, ny, nx] on 3-D grids (x fastest)."""
        if self.nz > 1:
            return (self.ncomp, self.nz, self.ny, self.nx)
        return (self.ncomp, self.ny, self.nx)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


@dataclass
class Workload:
    """A problem, its initial state and the number of implicit steps to take."""

    name: str
    problem: Problem
    u0: np.ndarray
    nsteps: int
    notes: str = ""
    extra: dict = field(default_factory=dict)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# --------------------------------------------------------------------------------------
# initial-condition generators
# --------------------------------------------------------------------------------------

def uniform_field(seed: int, shape, lo: float, hi: float) -> np.ndarray:
    """i.i.d. uniform[lo, hi] values (Section 3.2.3 uses uniform[-0.05, 0.05])."""
    return rng(seed).uniform(lo, hi, size=shape).astype(np.float64)


def zero_mean_uniform(seed: int, shape, half_width: float) -> np.ndarray:
    """i.i.d. uniform[-w, w], then the sample mean subtracted so the mean is exactly 0."""
    u = uniform_field(seed, shape, -half_width, half_width)
    return u - u.mean()


def _blur_reflect_1d(g: np.ndarray, axis: int, sigma: float, trunc: int) -> np.ndarray:
    taps = np.arange(-trunc, trunc + 1, dtype=np.float64)
    w = np.exp(-0.5 * (taps / sigma) ** 2)
    w /= w.sum()
    pad = [(0, 0)] * g.ndim
    pad[axis] = (trunc, trunc)
    gp = np.pad(g, pad, mode="symmetric")
    out = np.zeros_like(g)
    n = g.shape[axis]
    for t, wt in zip(range(2 * trunc + 1), w):
        sl = [slice(None)] * g.ndim
        sl[axis] = slice(t, t + n)
        out += wt * gp[tuple(sl)]
    return out


def smoothed_tanh(seed: int, ny: int, nx: int, sigma: float = 8.0, trunc: int = 32) -> np.ndarray:
    """tanh of seeded, Gaussian-smoothed white noise (reflective boundaries).

    g ~ N(0,1) i.i.d., blurred separably with a Gaussian of width ``sigma`` cells truncated at
    +-``trunc`` cells with mirror (Neumann-consistent) padding, then u0 = tanh(g / std(g)).
    """
    g = rng(seed).standard_normal((ny, nx))
    g = _blur_reflect_1d(g, 0, sigma, trunc)
    g = _blur_reflect_1d(g, 1, sigma, trunc)
    return np.tanh(g / g.std())


def gray_scott_patches(seed: int, n: int, npatch: int = 10, side_frac: float = 1 / 12.8,
                       u_in: float = 0.5, v_in: float = 0.25, noise: float = 0.01) -> np.ndarray:
    """u=1, v=0 background with ``npatch`` axis-aligned square patches (u=0.5, v=0.25) at
    seeded centres, wrapping periodically; then every value multiplied by (1 + noise*xi),
    xi ~ U[-1,1] i.i.d."""
    r = rng(seed)
    u = np.ones((n, n))
    v = np.zeros((n, n))
    side = max(1, int(round(n * side_frac)))
    for _ in range(npatch):
        ci, cj = r.integers(0, n, size=2)
        rows = (np.arange(side) + ci - side // 2) % n
        cols = (np.arange(side) + cj - side // 2) % n
        u[np.ix_(rows, cols)] = u_in
        v[np.ix_(rows, cols)] = v_in
    u *= 1.0 + noise * r.uniform(-1.0, 1.0, size=(n, n))
    v *= 1.0 + noise * r.uniform(-1.0, 1.0, size=(n, n))
    return np.stack([u, v])


def cell_centres(n: int, length: float, bc: str) -> np.ndarray:
    """Node coordinates along one axis: periodic nodes at j*h, Neumann at (j+1/2)*h, h=length/n."""
    h = length / n
    off = 0.5 if bc == "neumann" else 0.0
    return (np.arange(n) + off) * h


def cosine_mode(pb: Problem, kx: int, ky: int) -> np.ndarray:
    """One eigenmode of the grid Laplacian: cos(2 pi (kx j/nx + ky i/ny)) on periodic grids,
    cos(pi kx (j+1/2)/nx) cos(pi ky (i+1/2)/ny) on cell-centred Neumann grids."""
    j = np.arange(pb.nx)[None, :]
    i = np.arange(pb.ny)[:, None]
    if pb.bc == "periodic":
        m = np.cos(2 * np.pi * (kx * j / pb.nx + ky * i / pb.ny))
    else:
        m = np.cos(np.pi * kx * (j + 0.5) / pb.nx) * np.cos(np.pi * ky * (i + 0.5) / pb.ny)
    return np.broadcast_to(m, (pb.ncomp, pb.ny, pb.nx)).copy()


def seven_circles(n: int, node_offset: float = 0.0, mollifier_eps: float = 0.1) -> np.ndarray:
    """Cahn-Hilliard seven-circle initial data of Section 3.2.1 (Table 1), on [0,2pi)^2, at the
    periodic nodes (j + node_offset) h, h = 2 pi / n, with the mollifier width eps of that
    section (0.1)."""
    xs = np.array([np.pi / 2, np.pi / 4, np.pi / 2, np.pi, 3 * np.pi / 2, np.pi, 3 * np.pi / 2])
    ys = np.array([np.pi / 2, 3 * np.pi / 4, 5 * np.pi / 4, np.pi / 4, np.pi / 4, np.pi, 3 * np.pi / 2])
    rs = np.array([np.pi / 5, 2 * np.pi / 15, np.pi / 15, np.pi / 10, np.pi / 10, np.pi / 4, np.pi / 4])
    eps = mollifier_eps
    x = cell_centres(n, 2 * np.pi, "periodic") + node_offset * 2 * np.pi / n
    X, Y = np.meshgrid(x, x)
    u = -np.ones((n, n))
    for xi, yi, ri in zip(xs, ys, rs):
        s = np.sqrt((X - xi) ** 2 + (Y - yi) ** 2) - ri
        with np.errstate(divide="ignore", over="ignore"):
            u += np.where(s < 0, 2 * np.exp(-(eps ** 2) / np.where(s < 0, s, 1.0) ** 2), 0.0)
    return u[None]


def schnakenberg_initial(n: int, a_s: float = 0.1305, b_s: float = 0.7695) -> np.ndarray:
    """Schnakenberg initial data of Section 3.4.1: a perturbed equilibrium on [0,1]^2."""
    x = cell_centres(n, 1.0, "neumann")
    X, Y = np.meshgrid(x, x)
    u = a_s + b_s + 1e-3 * np.exp(-100 * ((X - 1 / 3) ** 2 + (Y - 0.5) ** 2))
    v = np.full_like(u, b_s / (a_s + b_s) ** 2)
    return np.stack([u, v])


# --------------------------------------------------------------------------------------
# the synthetic configurations
# --------------------------------------------------------------------------------------

def config_allen_cahn_periodic(n: int = 64, nsteps: int = 20, seed: int = 1000) -> Workload:
    """Allen-Cahn, periodic [0,2pi)^2, eps=0.1 with a=eps, b=1/eps (Section 3.1 scaling),
    dt=0.01, u0 ~ U[-0.05,0.05], stop on ||Res||_2 <= 1e-10 (plain FP64)."""
    eps = 0.1
    pb = Problem(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc="periodic", op="laplacian",
                 kind="allen_cahn", a=eps, b=1 / eps, dt=0.01, tau_u=1.0, tau_p=1.0,
                 tol=1e-10, tol_kind="res_abs")
    return Workload("allen_cahn_periodic_%d" % n, pb, uniform_field(seed, (1, n, n), -0.05, 0.05), nsteps)


def config_allen_cahn_periodic_3d(n: int = 128, nsteps: int = 20, seed: int = 6000) -> Workload:
    """Allen-Cahn on the serving mix's 3-D grid: periodic [0,2pi)^3 with n^3 points, the physics of
    the 64^2 configuration (a = eps = 0.1, b = 1/eps, dt = 0.01), u0 ~ U[-0.05, 0.05], each step
    solved to ||F||_2 <= 1e-11 ||U^k||_2."""
    eps = 0.1
    L = 2 * np.pi
    pb = Problem(nx=n, ny=n, nz=n, lx=L, ly=L, lz=L, bc="periodic", op="laplacian", kind="allen_cahn",
                 a=eps, b=1 / eps, dt=0.01, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
    return Workload("allen_cahn_periodic_%dx3" % n, pb, uniform_field(seed, pb.shape, -0.05, 0.05), nsteps)


def config_allen_cahn_periodic_8192(n: int = 8192, nsteps: int = 2, seed: int = 7000,
                                    fixed_iters: int = 200) -> Workload:
    """The roofline sweep: Allen-Cahn, periodic [0,2pi)^2 with n^2 points and the physics of the
    64^2 configuration (a = eps = 0.1, b = 1/eps, dt = 0.01), u0 ~ U[-0.05, 0.05] iid, and a
    fixed number of PDHG iterations per step (threshold 0: the stopping rule never fires, the
    step ends after max_iter = fixed_iters updates)."""
    eps = 0.1
    L = 2 * np.pi
    pb = Problem(nx=n, ny=n, lx=L, ly=L, bc="periodic", op="laplacian", kind="allen_cahn",
                 a=eps, b=1 / eps, dt=0.01, tau_u=1.0, tau_p=1.0, tol=0.0, tol_kind="res_abs",
                 max_iter=fixed_iters)
    return Workload("allen_cahn_periodic_%d" % n, pb, uniform_field(seed, (1, n, n), -0.05, 0.05), nsteps)


def config_allen_cahn_neumann(n: int = 1024, nsteps: int = 100, seed: int = 2000) -> Workload:
    """Allen-Cahn, Neumann [0,1]^2 cell-centred (h=1/n), eps=0.01 (a=eps, b=1/eps), dt=1e-4,
    u0 = tanh of smoothed noise (sigma = 8 cells), stop on ||F||_2 <= 1e-11 ||U^k||_2."""
    eps = 0.01
    pb = Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="neumann", op="laplacian", kind="allen_cahn",
                 a=eps, b=1 / eps, dt=1e-4, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
    return Workload("allen_cahn_neumann_%d" % n, pb, smoothed_tanh(seed, n, n)[None], nsteps)


def config_cahn_hilliard_split(n: int = 512, nsteps: int = 200, seed: int = 3000) -> Workload:
    """Cahn-Hilliard, periodic [0,1]^2, convex-concave split (U^3 implicit, -U explicit),
    eps=0.02 with a=eps^2, b=1 (Section 3.2 scaling), dt=1e-5, u0 zero-mean U[-0.1,0.1]."""
    eps = 0.02
    pb = Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="periodic", op="neg_biharmonic", kind="ch_split",
                 a=eps * eps, b=1.0, dt=1e-5, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
    return Workload("cahn_hilliard_split_%d" % n, pb, zero_mean_uniform(seed, (1, n, n), 0.1), nsteps)


def config_gray_scott(n: int = 2048, nsteps: int = 50, seed: int = 4000) -> Workload:
    """Two-species Gray-Scott, periodic [0,2.5)^2, Du=2e-5, Dv=1e-5, F=0.04, k=0.06, dt=1."""
    pb = Problem(nx=n, ny=n, lx=2.5, ly=2.5, bc="periodic", op="laplacian", kind="gray_scott",
                 p=(2e-5, 1e-5, 0.04, 0.06), dt=1.0, tau_u=0.9, tau_p=0.9, tol=1e-11,
                 tol_kind="f_rel")
    return Workload("gray_scott_%d" % n, pb, gray_scott_patches(seed, n), nsteps)


def config_schnakenberg(n: int = 128, nsteps: int = 10) -> Workload:
    """Schnakenberg system of Section 3.4.1: Neumann [0,1]^2, kappa=100, a=0.1305, b=0.7695,
    D1=0.05, D2=1, dt=1/5000, tau_u=tau_p=0.9, stop on ||Res_U||+||Res_V|| <= 1e-7."""
    pb = Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="neumann", op="laplacian", kind="schnakenberg",
                 p=(0.05, 1.0, 100.0, 0.1305, 0.7695), dt=1 / 5000, tau_u=0.9, tau_p=0.9,
                 tol=1e-7, tol_kind="res_abs")
    return Workload("schnakenberg_%d" % n, pb, schnakenberg_initial(n), nsteps)


def config_seven_circles(n: int = 128) -> Workload:
    """Cahn-Hilliard seven circles of Section 3.2.1: [0,2pi)^2, a=0.01, b=1, dt=1/200,
    tau_u=tau_p=0.5 (fully implicit)."""
    pb = Problem(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc="periodic", op="neg_biharmonic",
                 kind="ch_implicit", a=0.01, b=1.0, dt=1 / 200, tau_u=0.5, tau_p=0.5,
                 tol=1e-7, tol_kind="res_abs")
    return Workload("seven_circles_%d" % n, pb, seven_circles(n), 6000)


def fch_initial(n: int) -> np.ndarray:
    """Initial data of the sixth-order example of Section 3.3 (eq. 6th order initial) on [0,2pi)^2:
    u0 = 2 exp(sin x + sin y - 2) + 2.2 exp(-sin x - sin y - 2) - 1."""
    x = cell_centres(n, 2 * np.pi, "periodic")
    X, Y = np.meshgrid(x, x)
    s = np.sin(X) + np.sin(Y)
    return (2 * np.exp(s - 2) + 2.2 * np.exp(-s - 2) - 1)[None]


def config_fch(n: int = 128) -> Workload:
    """Functionalized (sixth-order) Cahn-Hilliard of Section 3.3: [0,2pi)^2 periodic, eps = 0.18
    (a = eps^2, b = 1), dt = 1/1000, tau_u = tau_p = 0.58, delta = 0.5e-5, 20000 steps."""
    pb = Problem(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc="periodic", op="functionalized", kind="fch",
                 a=0.18 ** 2, b=1.0, dt=1e-3, tau_u=0.58, tau_p=0.58, tol=0.5e-5, tol_kind="res_abs")
    return Workload("fch_%d" % n, pb, fch_initial(n), 20000)


def scaled(w: Workload, n: int, nsteps: int | None = None) -> Workload:
    """The same physics on an n x n grid (same domain, so h changes with n)."""
    pb = w.problem.replace(nx=n, ny=n)
    name = w.name.rsplit("_", 1)[0] + "_%d" % n
    return Workload(name, pb, None, nsteps if nsteps is not None else w.nsteps, w.notes)


def workload_small(name: str, n: int, nsteps: int, seed: int = 7) -> Workload:
    """A configuration's physics on a reduced n x n grid with its own initial-data recipe."""
    if name == "allen_cahn_periodic":
        return config_allen_cahn_periodic(n, nsteps, seed)
    if name == "allen_cahn_neumann":
        w = config_allen_cahn_neumann(n, nsteps, seed)
        return w
    if name == "cahn_hilliard_split":
        return config_cahn_hilliard_split(n, nsteps, seed)
    if name == "gray_scott":
        return config_gray_scott(n, nsteps, seed)
    if name == "schnakenberg":
        return config_schnakenberg(n, nsteps)
    raise KeyError(name)


# --------------------------------------------------------------------------------------
# serving mix
# --------------------------------------------------------------------------------------

SERVING_SIDES = (64, 128, 256, 512, 1024)
SERVING_CUBE = 128      # the mix's 3-D grid, 128^3


def serving_requests(n: int, seed: int = 5000, min_steps: int = 10, max_steps: int = 50,
                     sides=SERVING_SIDES, tol: float = 1e-6, cube=SERVING_CUBE):
    """The serving mix: n seeded requests, each an Allen-Cahn (physics of the 64^2 periodic
    configuration, domain [0,2pi)^d) or Cahn-Hilliard convex-split (physics of the 512^2
    configuration, domain [0,1]^d) run of min_steps..max_steps implicit steps, periodic or
    Neumann 50/50, each step solved to ||F||_2 <= tol ||U^k||_2, on a grid drawn uniformly from
    the square grids `sides`^2 and the cube `cube`^3 (cube = None: square grids only).  The 3-D
    draw comes from its own seeded stream (probability 1 / (len(sides) + 1) per request), so the
    square-grid requests are the same with and without the cube.  Returns a list of
    (Problem, u0, nsteps)."""
    r = rng(seed)
    r3 = rng(seed + 7919)
    out = []
    for k in range(n):
        side = int(r.choice(sides))
        bc = "periodic" if r.random() < 0.5 else "neumann"
        steps = int(r.integers(min_steps, max_steps + 1))
        three = cube is not None and r3.random() < 1.0 / (len(sides) + 1)
        g = dict(nx=cube, ny=cube, nz=cube) if three else dict(nx=side, ny=side)
        if r.random() < 0.5:
            L = 2 * np.pi
            pb = Problem(lx=L, ly=L, lz=L, bc=bc, op="laplacian",
                         kind="allen_cahn", a=0.1, b=10.0, dt=0.01, tau_u=1.0, tau_p=1.0,
                         tol=tol, tol_kind="f_rel", **g)
            u0 = uniform_field(seed + 1 + k, pb.shape, -0.05, 0.05)
        else:
            pb = Problem(lx=1.0, ly=1.0, lz=1.0, bc=bc, op="neg_biharmonic",
                         kind="ch_split", a=4e-4, b=1.0, dt=1e-5, tau_u=1.0, tau_p=1.0,
                         tol=tol, tol_kind="f_rel", **g)
            u0 = zero_mean_uniform(seed + 1 + k, pb.shape, 0.1)
        out.append((pb, u0, steps))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 5999) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process of the given rate."""
    return np.cumsum(rng(seed).exponential(1.0 / rate, size=n))
