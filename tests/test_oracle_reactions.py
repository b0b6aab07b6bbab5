"""Pins of the oracle's reaction terms against the PDEs they discretise, CPU only.

The dense pins (tests/test_oracle_operators.py, test_oracle_iteration.py) fix the solve and the
adjoint given F.  These tests fix F itself from outside the oracle: each writes the reaction of
its PDE from the equation (Gray-Scott in its standard form, Schnakenberg as printed in Section
3.4.1, Allen-Cahn eq. AC equ, Cahn-Hilliard eq. CH equ with its convex-concave split) and checks
the oracle's PDHG step against
  * spatially uniform states, where every Laplacian vanishes and one implicit step is a
    backward-Euler step of the reaction ODE, solved here by a 2x2 (or scalar) Newton iteration;
  * uniform steady states of the PDE, which every implicit step must leave unchanged;
  * one small Fourier or DCT mode on a uniform steady state, whose amplitude after one step is
    fixed by the linearised PDE in closed form: a_{k+1} = m(mu) a_k with mu the eigenvalue of
    -Lap of the mode, up to O(eps^2) relative (the quadratic terms land in the mean and in the
    doubled mode, not in the mode itself).
A sign, index or coefficient mistake in any reaction term (u v^2 against F(1 - u), the split's
+b dt Lap U^k, D_u against D_v) moves one of these by far more than its tolerance.  Every test
runs against both oracles (numpy and C++).
"""
import math

import numpy as np
import pytest

from oracle import cpp_oracle, rd_oracle
from paper_2305_03945_gb300 import workloads as WL


@pytest.fixture(params=["numpy", "cpp"])
def O(request):
    """Both oracles: the numpy restatement and the plain C++ one."""
    if request.param == "cpp":
        cpp_oracle.set_threads(1)
        yield cpp_oracle
        cpp_oracle.set_threads(0)
    else:
        yield rd_oracle

TIGHT = dict(tol=1e-14, tol_kind="f_rel", max_iter=20000)


def _uniform(pb, vals):
    return np.stack([np.full((pb.ny, pb.nx), v) for v in vals])


def _newton2(G, J, x0, tol=1e-15, it=60):
    x = np.array(x0, dtype=np.float64)
    for _ in range(it):
        g = np.array(G(*x))
        if np.max(np.abs(g)) <= tol:
            return x
        x = x - np.linalg.solve(np.array(J(*x)), g)
    raise RuntimeError("2x2 Newton did not converge")


def _mode(pb, kx, ky):
    """A Laplacian eigenmode and its eigenvalue mu of -Lap, written from the stencil's closed
    form: periodic e.v. (4/h^2) sin^2(pi k/N), Neumann cell-centred (4/h^2) sin^2(pi k/(2N))."""
    hx, hy = pb.lx / pb.nx, pb.ly / pb.ny
    j = np.arange(pb.nx)[None, :]
    i = np.arange(pb.ny)[:, None]
    if pb.bc == "periodic":
        phi = np.cos(2 * np.pi * (kx * j / pb.nx + ky * i / pb.ny))
        mu = 4 / hx ** 2 * math.sin(math.pi * kx / pb.nx) ** 2 + 4 / hy ** 2 * math.sin(math.pi * ky / pb.ny) ** 2
    else:
        phi = np.cos(np.pi * kx * (j + 0.5) / pb.nx) * np.cos(np.pi * ky * (i + 0.5) / pb.ny)
        mu = (4 / hx ** 2 * math.sin(math.pi * kx / (2 * pb.nx)) ** 2
              + 4 / hy ** 2 * math.sin(math.pi * ky / (2 * pb.ny)) ** 2)
    return phi, mu


def _amplitude(field, phi):
    return float(np.sum(field * phi) / np.sum(phi * phi))


# ------------------------------------------------------------------------------------------
# Gray-Scott: u_t = Du Lap u - u v^2 + F (1 - u),  v_t = Dv Lap v + u v^2 - (F + k) v
# ------------------------------------------------------------------------------------------

def _gs(bc, n=16, dt=1.0, p=(2e-5, 1e-5, 0.04, 0.06)):
    return WL.Problem(nx=n, ny=n, lx=2.5, ly=2.5, bc=bc, op="laplacian", kind="gray_scott", p=p, dt=dt,
                      tau_u=0.9, tau_p=0.9, **TIGHT)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("dt", [0.5, 1.0])
def test_gray_scott_uniform_step_is_the_ode_step(bc, dt, O):
    pb = _gs(bc, dt=dt)
    Du, Dv, Ff, k = pb.p
    uk, vk = 0.7, 0.2
    G = lambda u, v: (u - uk - dt * (-u * v * v + Ff * (1 - u)), v - vk - dt * (u * v * v - (Ff + k) * v))
    J = lambda u, v: ((1 + dt * (v * v + Ff), 2 * dt * u * v), (-dt * v * v, 1 - dt * (2 * u * v - (Ff + k))))
    us, vs = _newton2(G, J, (uk, vk))
    U, info = O.pdhg_step(pb, _uniform(pb, (uk, vk)))
    assert info["status"] == O.OK
    assert np.max(np.abs(U[0] - us)) <= 1e-12 and np.max(np.abs(U[1] - vs)) <= 1e-12


def test_gray_scott_steady_states_are_fixed_points(O):
    """(1, 0) and, for F = 0.04, k = 0.05, the two uniform roots of u v = F + k,
    F (1 - u) = (F + k) v (a quadratic in v) are steady: F(U) = 0 at U = U^k."""
    pb = _gs("periodic", p=(2e-5, 1e-5, 0.04, 0.05))
    Ff, k = pb.p[2], pb.p[3]
    s = Ff + k
    disc = Ff * Ff - 4 * Ff * s * s
    states = [(1.0, 0.0)] + [(s / v, v) for v in ((Ff + r) / (2 * s) for r in (math.sqrt(disc), -math.sqrt(disc)))]
    for u, v in states:
        X = _uniform(pb, (u, v))
        assert np.max(np.abs(O.residual(pb, X, X))) <= 1e-15
        U, info = O.pdhg_step(pb, X)
        assert info["status"] == O.OK and np.max(np.abs(U - X)) <= 1e-14


@pytest.mark.parametrize("bc,kx,ky", [("periodic", 3, 1), ("neumann", 2, 5)])
def test_gray_scott_mode_on_the_trivial_state_decays_per_species(bc, kx, ky, O):
    """Around (1, 0) the linearised step is u^ <- u^ / (1 + dt (Du mu + F)) and
    v^ <- v^ / (1 + dt (Dv mu + F + k)): each species' own diffusion and linear reaction."""
    pb = _gs(bc, dt=1.0, p=(2e-3, 1e-3, 0.04, 0.06))
    Du, Dv, Ff, k = pb.p
    phi, mu = _mode(pb, kx, ky)
    e = 1e-5
    X = np.stack([1 + e * phi, 0.5 * e * phi])
    U, info = O.pdhg_step(pb, X)
    assert info["status"] == O.OK
    au, av = _amplitude(U[0] - 1, phi), _amplitude(U[1], phi)
    assert au == pytest.approx(e / (1 + pb.dt * (Du * mu + Ff)), rel=1e-8)
    assert av == pytest.approx(0.5 * e / (1 + pb.dt * (Dv * mu + Ff + k)), rel=1e-8)


# ------------------------------------------------------------------------------------------
# Schnakenberg (Section 3.4.1): u_t = D1 Lap u + kappa (a - u + u^2 v), v_t = D2 Lap v + kappa (b - u^2 v)
# ------------------------------------------------------------------------------------------

def _sch(n=8, dt=1 / 5000):
    return WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="neumann", op="laplacian", kind="schnakenberg",
                      p=(0.05, 1.0, 100.0, 0.1305, 0.7695), dt=dt, tau_u=0.9, tau_p=0.9, **TIGHT)


def test_schnakenberg_equilibrium_is_a_fixed_point(O):
    """The equilibrium (a + b, b / (a + b)^2) that Section 3.4.1 perturbs."""
    pb = _sch()
    a_s, b_s = pb.p[3], pb.p[4]
    X = _uniform(pb, (a_s + b_s, b_s / (a_s + b_s) ** 2))
    assert np.max(np.abs(O.residual(pb, X, X))) <= 1e-15
    U, info = O.pdhg_step(pb, X)
    assert info["status"] == O.OK and np.max(np.abs(U - X)) <= 1e-14


@pytest.mark.parametrize("dt", [1 / 5000, 1 / 1000])
def test_schnakenberg_uniform_step_is_the_ode_step(dt, O):
    pb = _sch(dt=dt)
    kap, a_s, b_s = pb.p[2], pb.p[3], pb.p[4]
    uk, vk = 1.1, 0.5
    G = lambda u, v: (u - uk - dt * kap * (a_s - u + u * u * v), v - vk - dt * kap * (b_s - u * u * v))
    J = lambda u, v: ((1 + dt * kap * (1 - 2 * u * v), -dt * kap * u * u), (2 * dt * kap * u * v, 1 + dt * kap * u * u))
    us, vs = _newton2(G, J, (uk, vk))
    U, info = O.pdhg_step(pb, _uniform(pb, (uk, vk)))
    assert info["status"] == O.OK
    assert np.max(np.abs(U[0] - us)) <= 1e-12 and np.max(np.abs(U[1] - vs)) <= 1e-12


# ------------------------------------------------------------------------------------------
# Allen-Cahn (eq. AC equ): u_t = a Lap u - b (u^3 - u)
# ------------------------------------------------------------------------------------------

def _ac(bc, n=16, dt=0.01):
    return WL.Problem(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc=bc, op="laplacian", kind="allen_cahn",
                      a=0.1, b=10.0, dt=dt, tau_u=1.0, tau_p=1.0, **TIGHT)


@pytest.mark.parametrize("uk", [0.3, -0.8, 1.2])
def test_allen_cahn_uniform_step_is_the_ode_step(uk, O):
    pb = _ac("periodic").replace(tau_u=0.7, tau_p=0.7)
    us = _newton2(lambda u, v: (u - uk + pb.dt * pb.b * (u ** 3 - u), v),
                  lambda u, v: ((1 + pb.dt * pb.b * (3 * u * u - 1), 0.0), (0.0, 1.0)), (uk, 0.0))[0]
    U, info = O.pdhg_step(pb, _uniform(pb, (uk,)))
    assert info["status"] == O.OK and np.max(np.abs(U - us)) <= 1e-12


@pytest.mark.parametrize("bc,kx,ky", [("periodic", 2, 3), ("neumann", 4, 1)])
@pytest.mark.parametrize("ubar", [0.0, 1.0, -1.0])
def test_allen_cahn_mode_on_a_steady_state(bc, kx, ky, ubar, O):
    """Around the uniform steady states u = 0, +-1: u^ <- u^ / (1 + dt (a mu + b (3 u^2 - 1)))."""
    pb = _ac(bc, dt=0.005)
    phi, mu = _mode(pb, kx, ky)
    e = 1e-6
    U, info = O.pdhg_step(pb, (ubar + e * phi)[None])
    assert info["status"] == O.OK
    m = 1 / (1 + pb.dt * (pb.a * mu + pb.b * (3 * ubar * ubar - 1)))
    assert _amplitude(U[0] - ubar, phi) == pytest.approx(e * m, rel=1e-8)


# ------------------------------------------------------------------------------------------
# Cahn-Hilliard (eq. CH equ): u_t = -a Lap^2 u + b Lap W'(u); fully implicit, and the convex-
# concave split with u^3 implicit and -u explicit
# ------------------------------------------------------------------------------------------

def _ch(kind, bc, n=16, dt=1e-5):
    return WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc=bc, op="neg_biharmonic", kind=kind, a=4e-4, b=1.0, dt=dt,
                      tau_u=1.0, tau_p=1.0, **TIGHT)


@pytest.mark.parametrize("bc,kx,ky", [("periodic", 1, 2), ("neumann", 3, 2)])
@pytest.mark.parametrize("ubar", [0.0, 0.45])
def test_cahn_hilliard_split_mode(bc, kx, ky, ubar, O):
    """Split step on u = ubar + eps phi:
    (1 + a dt mu^2 + 3 b dt ubar^2 mu) u^ = (1 + b dt mu) u^k^  (ubar = 0 isolates the explicit
    +b dt Lap U^k term, ubar != 0 the implicit U^3 term); the mean stays ubar."""
    pb = _ch("ch_split", bc)
    phi, mu = _mode(pb, kx, ky)
    e = 1e-5
    U, info = O.pdhg_step(pb, (ubar + e * phi)[None])
    assert info["status"] == O.OK
    m = (1 + pb.b * pb.dt * mu) / (1 + pb.a * pb.dt * mu * mu + 3 * pb.b * pb.dt * ubar * ubar * mu)
    assert _amplitude(U[0] - ubar, phi) == pytest.approx(e * m, rel=1e-8)
    assert abs(U[0].mean() - ubar) <= 1e-14


@pytest.mark.parametrize("bc,kx,ky", [("periodic", 1, 2), ("neumann", 3, 2)])
@pytest.mark.parametrize("ubar", [0.0, 0.45, 0.9])
def test_cahn_hilliard_implicit_mode(bc, kx, ky, ubar, O):
    """Fully implicit step: (1 + a dt mu^2 + b dt (3 ubar^2 - 1) mu) u^ = u^k^."""
    pb = _ch("ch_implicit", bc)
    phi, mu = _mode(pb, kx, ky)
    e = 1e-5
    U, info = O.pdhg_step(pb, (ubar + e * phi)[None])
    assert info["status"] == O.OK
    m = 1 / (1 + pb.a * pb.dt * mu * mu + pb.b * pb.dt * (3 * ubar * ubar - 1) * mu)
    assert _amplitude(U[0] - ubar, phi) == pytest.approx(e * m, rel=1e-8)
    assert abs(U[0].mean() - ubar) <= 1e-14
