"""Pins of the oracle's PDHG iteration (CPU only): closed-form linear theory, direct solves,
dense Newton, invariants and the iteration counts the paper prints."""
import json
import math
import os

import numpy as np
import pytest

from oracle import dense, rd_oracle as O, theory
from paper_2305_03945_gb300 import workloads as WL

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def _mode_problem(bc, op, tau_u, tau_p, precond="linear", omega=1.0, n=16, tol=0.0, max_iter=40):
    a = 0.3 if op == "laplacian" else 2e-3
    return WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc=bc, op=op, kind="none", dt=1e-2, a=a,
                      tau_u=tau_u, tau_p=tau_p, omega=omega, precond=precond, tol=tol,
                      tol_kind="res_abs", max_iter=max_iter)


def _mode_alpha(pb, kx, ky):
    h = 1.0 / pb.nx
    d = 1 if pb.bc == "periodic" else 2
    mu = 4 / h ** 2 * (math.sin(math.pi * kx / (d * pb.nx)) ** 2 + math.sin(math.pi * ky / (d * pb.ny)) ** 2)
    return 1 + pb.dt * pb.a * (mu if pb.op == "laplacian" else mu * mu)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("op", ["laplacian", "neg_biharmonic"])
@pytest.mark.parametrize("taus,omega,precond", [
    ((1.0, 1.0), 1.0, "linear"),      # nilpotent: exact in two iterations
    ((0.7, 0.7), 1.0, "linear"),      # t = 0.49: rate sqrt(0.51)
    ((0.5, 1.6), 1.0, "linear"),      # unequal steps, t = 0.8
    ((0.9, 0.9), 0.5, "linear"),      # omega other than 1
    ((0.01, 0.01), 1.0, "none"),      # G = I: Theorem 1 with lam = alpha (all modes stable)
])
def test_single_mode_history_matches_recurrence(bc, op, taus, omega, precond):
    """On one Laplacian eigenmode with the reaction off, the oracle's residual history equals
    the scalar G-prox recurrence of Appendix A (p, e per mode) to 1e-12 relative."""
    tau_u, tau_p = taus
    pb = _mode_problem(bc, op, tau_u, tau_p, precond, omega, max_iter=25)
    kx, ky = 3, 2
    m = WL.cosine_mode(pb, kx, ky)
    alpha = _mode_alpha(pb, kx, ky)
    g = alpha ** 2 if precond == "linear" else 1.0
    e0 = 1 - 1 / alpha                         # U_0 = U^k = m, U_* = m / alpha
    U, info = O.pdhg_step(pb, m, history=True)
    want = np.abs(theory.single_mode_residuals(alpha, g, tau_u, tau_p, omega, e0, 25))
    want = want * np.linalg.norm(m) / pb.dt
    got = info["history"]
    n = min(len(got), len(want))
    scale = want[0]
    assert np.max(np.abs(got[:n] - want[:n])) <= 1e-12 * scale + 1e-14
    assert info["iterations"] == n - 1


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_unit_steps_are_nilpotent(bc):
    """With G = A^2 (reaction off) every preconditioned mode has lam = 1, so tau_u tau_p = 1 makes
    D_k nilpotent: random data are solved exactly after two updates (Corollary 1, App. A)."""
    pb = _mode_problem(bc, "laplacian", 1.0, 1.0, tol=1e-13 * 1e4, max_iter=10)
    uk = WL.rng(1).standard_normal(pb.shape)
    U, info = O.pdhg_step(pb, uk, history=True)
    h = info["history"]
    assert info["status"] == O.OK and info["iterations"] == 2
    assert h[1] > 1e-3 * h[0] and h[2] <= 1e-13 * h[0]


def test_random_data_follow_preconditioned_iteration_matrix():
    """Corollary 1: with G = A^2 every mode sees the same 2x2 matrix D (lam = 1), so for ANY
    data the residual history is r_n = |(D^n)_11| r_0, and its modulus decays like
    sqrt(1 - t), t = tau_u tau_p < 1 (Appendix A)."""
    tau_u, tau_p = 0.8, 0.8
    t = tau_u * tau_p
    pb = _mode_problem("periodic", "laplacian", tau_u, tau_p, max_iter=40)
    uk = WL.rng(2).standard_normal(pb.shape)
    _, info = O.pdhg_step(pb, uk, history=True)
    h = info["history"]
    D = theory.iteration_matrix(tau_u, tau_p, 1.0)
    Dn = np.eye(2)
    for n in range(len(h)):
        assert abs(h[n] - abs(Dn[0, 0]) * h[0]) <= 1e-11 * h[0]
        Dn = D @ Dn
    assert abs(max(abs(np.linalg.eigvals(D))) - math.sqrt(1 - t)) < 1e-12


def test_steps_beyond_four_thirds_diverge():
    """tau_u tau_p = 1.4 > 4/3 (Theorem 1): the iteration blows up and is reported DIVERGED."""
    pb = _mode_problem("periodic", "laplacian", 1.4, 1.0, max_iter=100000)
    uk = WL.rng(3).standard_normal(pb.shape)
    _, info = O.pdhg_step(pb, uk)
    assert info["status"] == O.DIVERGED
    assert GOLDEN["theorem1"]["divergence_bound"] < 1.4


def test_rate_function_and_bound():
    """f(t) of Appendix A equals the spectral radius of D_k; f(0) = f(4/3) = 1, min at t = 1."""
    for t in np.linspace(0.01, 1.6, 40):
        D = theory.iteration_matrix(math.sqrt(t), math.sqrt(t), 1.0)
        rho = max(abs(np.linalg.eigvals(D)))
        assert abs(rho - theory.rate(t)) < 1e-7
    assert abs(theory.rate(4 / 3) - 1) < 1e-12 and theory.rate(1.0) == 0.0


@pytest.mark.parametrize("kappa", [1.2, 1.5, 3.0, 10.0, 100.0])  # kappa^2 >= 4/3: the branch of eq. (equation eta)
def test_eta_gamma_closed_forms(kappa):
    """Remark 2: eta_* solves sqrt(1 - eta/kappa^2) = eta - 1 + sqrt(eta^2 - eta) on [1, 4/3)
    (root found numerically by bisection here) and gamma_* = sqrt(1 - eta_*/kappa^2)."""
    g = lambda e: math.sqrt(1 - e / kappa ** 2) - (e - 1 + math.sqrt(e * e - e))
    lo, hi = 1.0, 4 / 3
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0:
            lo = mid
        else:
            hi = mid
    assert abs(theory.eta_star(kappa) - lo) < 1e-9
    assert 1.0 <= theory.eta_star(kappa) < 4 / 3
    assert abs(theory.gamma_star(kappa) - math.sqrt(1 - lo / kappa ** 2)) < 1e-9
    # the optimum balances the extreme modes
    assert abs(theory.rate(lo / kappa ** 2) - theory.rate(lo)) < 1e-7


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("op", ["laplacian", "neg_biharmonic"])
def test_reaction_off_step_is_direct_solve(bc, op):
    """Reaction off: one converged PDHG step equals the dense direct solve of A_lin u = u^n."""
    pb = _mode_problem(bc, op, 0.9, 0.9, tol=1e-12, max_iter=500)
    uk = WL.rng(4).standard_normal(pb.shape)
    U, info = O.pdhg_step(pb, uk)
    A = dense.linear_part(pb)[0]
    want = np.linalg.solve(A, uk.ravel())
    assert info["status"] == O.OK
    assert np.max(np.abs(U.ravel() - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_single_mode_decays_at_closed_form_rate(bc):
    """A single mode decays by exactly 1/(1 + h_t a mu) per implicit step; after 20 steps to 1e-12."""
    pb = _mode_problem(bc, "laplacian", 1.0, 1.0, tol=1e-14, max_iter=50).replace(tol_kind="f_rel")
    kx, ky = 1, 1
    m = WL.cosine_mode(pb, kx, ky)
    U, infos = O.solve(pb, m, 20)
    alpha = _mode_alpha(pb, kx, ky)
    assert all(i["status"] == O.OK for i in infos)
    assert np.max(np.abs(U - m / alpha ** 20)) <= 1e-12 * np.max(np.abs(m / alpha ** 20))


NEWTON_CASES = [
    ("allen_cahn", "laplacian", (), "periodic"),
    ("allen_cahn", "laplacian", (), "neumann"),
    ("ch_implicit", "neg_biharmonic", (), "periodic"),
    ("ch_implicit", "neg_biharmonic", (), "neumann"),
    ("ch_split", "neg_biharmonic", (), "periodic"),
    ("ch_split", "neg_biharmonic", (), "neumann"),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic"),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695), "neumann"),
    ("fch", "functionalized", (), "periodic"),
    ("fch", "functionalized", (), "neumann"),
]


def _newton_problem(kind, op, p, bc):
    if kind == "fch":   # Section 3.3's parameters on a 16^2 grid of [0,2pi]^2: eps = 0.18, h_t = 1e-3
        return WL.Problem(nx=16, ny=16, lx=2 * np.pi, ly=2 * np.pi, bc=bc, op=op, kind=kind, dt=1e-3,
                          a=0.18 ** 2, b=1.0, tau_u=0.58, tau_p=0.58, tol=1e-14, tol_kind="f_rel",
                          max_iter=20000)
    ch = op == "neg_biharmonic"
    return WL.Problem(nx=16, ny=16, lx=1.0, ly=1.0, bc=bc, op=op, kind=kind, p=p,
                      dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.02, b=1.0 if ch else 30.0,
                      tau_u=0.9, tau_p=0.9, tol=1e-14, tol_kind="f_rel", max_iter=5000)


def _newton_input(kind, n=16):
    r = WL.rng(21)
    if kind == "gray_scott":
        return np.stack([1 - 0.5 * r.random((n, n)), 0.25 * r.random((n, n))])
    if kind == "schnakenberg":
        return WL.schnakenberg_initial(n) * (1 + 0.05 * r.uniform(-1, 1, (2, n, n)))
    return r.uniform(-0.8, 0.8, (1, n, n))


@pytest.mark.parametrize("kind,op,p,bc", NEWTON_CASES)
def test_nonlinear_step_matches_dense_newton(kind, op, p, bc):
    """16x16: the converged PDHG step equals a dense Newton solve (own dense F and Jacobian,
    LU) to 1e-10 max relative error."""
    pb = _newton_problem(kind, op, p, bc)
    uk = _newton_input(kind)
    U, info = O.pdhg_step(pb, uk)
    Un = dense.newton(pb, uk)
    assert info["status"] == O.OK
    assert np.max(np.abs(U - Un)) <= 1e-10 * np.max(np.abs(Un))


@pytest.mark.parametrize("kind", ["ch_implicit", "ch_split"])
@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_cahn_hilliard_conserves_mass(kind, bc):
    """Sum Lap(.) = 0 on both grids, so a converged CH step keeps h^2 sum U to 1e-12."""
    w = WL.config_cahn_hilliard_split(32, 5, seed=9)
    pb = w.problem.replace(kind=kind, bc=bc, tol=1e-13)
    U = w.u0 + 0.3
    m0 = O.mass(pb, U)
    for _ in range(5):
        Un, info = O.pdhg_step(pb, U)
        assert info["status"] == O.OK
        assert abs(O.mass(pb, Un) - O.mass(pb, U)) <= 1e-12
        U = Un
    assert abs(O.mass(pb, U) - m0) <= 5e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_allen_cahn_energy_decreases_and_max_principle(bc):
    """Backward Euler AC with h_t <= 2/b: discrete energy non-increasing; |U| <= 1 kept."""
    eps = 0.05
    pb = WL.Problem(nx=32, ny=32, lx=1.0, ly=1.0, bc=bc, op="laplacian", kind="allen_cahn",
                    a=eps, b=1 / eps, dt=0.005, tau_u=0.8, tau_p=0.8, tol=1e-12, tol_kind="f_rel")
    assert pb.dt <= 2 / pb.b
    U = WL.uniform_field(8, pb.shape, -1.0, 1.0)
    E = O.ac_energy(pb, U)
    for _ in range(10):
        U, info = O.pdhg_step(pb, U)
        assert info["status"] == O.OK
        En = O.ac_energy(pb, U)
        assert En <= E + 1e-12 * abs(E)
        assert np.max(np.abs(U)) <= 1 + 1e-12
        E = En


def test_reflection_symmetry_preserved():
    """Data symmetric under x -> -x (periodic index j -> -j mod N) stay symmetric."""
    w = WL.config_allen_cahn_periodic(32, 3, seed=5)
    u = w.u0[0]
    u = 0.5 * (u + u[:, (-np.arange(32)) % 32])
    U, infos = O.solve(w.problem, u[None], 3)
    assert np.max(np.abs(U[0] - U[0][:, (-np.arange(32)) % 32])) <= 1e-13


def test_paper_allen_cahn_circle_iterations_below_200():
    """Section 3.1.1: shrinking circle, tau = 0.5, delta = 1e-7, fewer than 200 iterations."""
    g = GOLDEN["allen_cahn_circle"]
    n = g["n"]
    pb = WL.Problem(nx=n, ny=n, lx=g["side"], ly=g["side"], bc="periodic", op="laplacian",
                    kind="allen_cahn", a=g["eps"], b=1 / g["eps"], dt=g["dt"], tau_u=g["tau"],
                    tau_p=g["tau"], tol=g["delta"], tol_kind="res_abs")
    x = -g["side"] / 2 + np.arange(n) * g["side"] / n
    X, Y = np.meshgrid(x, x)
    u0 = np.where(X ** 2 + Y ** 2 < g["radius"] ** 2, 1.0, -1.0)[None]
    _, infos = O.solve(pb, u0, 3)
    its = [i["iterations"] for i in infos]
    assert all(i["status"] == O.OK for i in infos)
    assert max(its) < g["max_iterations"] and min(its) > 100


def test_paper_allen_cahn_two_disks_at_most_200_iterations():
    """Section 3.1.1, second example: the symmetric difference of two overlapping disks on
    [0, 0.5]^2 (nodes at j h), tau = 0.5: no more than 200 iterations per step (the numpy oracle:
    100 points a side is not a power of two)."""
    g = GOLDEN["allen_cahn_two_disks"]
    n = g["n"]
    pb = WL.Problem(nx=n, ny=n, lx=g["side"], ly=g["side"], bc="periodic", op="laplacian",
                    kind="allen_cahn", a=g["eps"], b=1 / g["eps"], dt=g["dt"], tau_u=g["tau"],
                    tau_p=g["tau"], tol=g["delta"], tol_kind="res_abs")
    x = np.arange(n) * g["side"] / n
    X, Y = np.meshgrid(x, x)
    inside = [(X - cx) ** 2 + (Y - cy) ** 2 < g["radius"] ** 2 for cx, cy in g["centres"]]
    u0 = np.where(inside[0] ^ inside[1], 1.0, -1.0)[None]
    _, infos = O.solve(pb, u0, 3)
    assert all(i["status"] == O.OK for i in infos)
    assert max(i["iterations"] for i in infos) <= g["max_iterations"]


def test_allen_cahn_circle_shrinks_by_its_curvature_law():
    """Section 3.1.1's shrinking circle: with a = eps, b = 1/eps the zero level set of Allen-Cahn
    moves with normal speed eps times its curvature, so a circle's radius follows
    r(t)^2 = r0^2 - 2 eps t (asymptotically in eps; a sanity band).  On [-0.25, 0.25)^2 with
    eps = 0.02, 64 points a side (h < eps) and h_t = 2e-3, the radius of the area {u > 0} after 100
    implicit steps (t = 0.2, r from 0.2 to 0.179) stays within 2% of the law; a mistaken scaling
    of either term (a = eps^2, or b = 1 / eps^2) moves it by far more.  The C++ oracle on all host
    cores (the numpy one takes about 15 s here)."""
    from oracle import cpp_oracle
    n, side, eps, r0, dt, steps = 64, 0.5, 0.02, 0.2, 2e-3, 100
    pb = WL.Problem(nx=n, ny=n, lx=side, ly=side, bc="periodic", op="laplacian", kind="allen_cahn",
                    a=eps, b=1 / eps, dt=dt, tau_u=0.5, tau_p=0.5, tol=1e-7, tol_kind="res_abs")
    x = -side / 2 + np.arange(n) * side / n
    X, Y = np.meshgrid(x, x)
    u0 = np.where(X ** 2 + Y ** 2 < r0 ** 2, 1.0, -1.0)[None]
    cpp_oracle.set_threads(0)
    U, infos = cpp_oracle.solve(pb, u0, steps)
    assert len(infos) == steps and all(i["status"] == cpp_oracle.OK for i in infos)
    h = side / n
    r = math.sqrt(np.sum(U[0] > 0) * h * h / math.pi)
    law = math.sqrt(r0 ** 2 - 2 * eps * steps * dt)
    assert abs(r / law - 1) <= 0.02, (r, law)


def test_paper_schnakenberg_about_30_iterations():
    """Section 3.4.1: about 30 PDHG iterations per time step (band 20..40)."""
    w = WL.config_schnakenberg(GOLDEN["schnakenberg"]["n"], 3)
    _, infos = O.solve(w.problem, w.u0, 3)
    assert all(20 <= i["iterations"] <= 40 for i in infos)


def test_not_converged_status():
    w = WL.config_allen_cahn_periodic(16, 1)
    U, info = O.pdhg_step(w.problem.replace(max_iter=3), w.u0)
    assert info["status"] == O.NOT_CONVERGED and info["iterations"] == 3


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_non_finite_state_diverges_before_any_update(bad):
    """A NaN or Inf in U^k makes the first measure non-finite: DIVERGED with 0 updates, in both
    oracles, and the returned U is U^k."""
    from oracle import cpp_oracle
    w = WL.config_allen_cahn_periodic(16, 1)
    uk = w.u0.copy()
    uk[0, 3, 5] = bad
    for M in (O, cpp_oracle):
        with np.errstate(invalid="ignore", over="ignore"):
            U, info = M.pdhg_step(w.problem.replace(tol_kind="f_rel", tol=1e-11), uk)
        assert info["status"] == M.DIVERGED and info["iterations"] == 0
        assert np.array_equal(U, uk, equal_nan=True)


def test_zero_state_converges_immediately():
    w = WL.config_allen_cahn_periodic(16, 1)
    U, info = O.pdhg_step(w.problem.replace(tol_kind="f_rel", tol=1e-11), np.zeros((1, 16, 16)))
    assert info["status"] == O.OK and info["iterations"] == 0


@pytest.mark.parametrize("tol_kind,tol", [("res_abs", 1e-8), ("f_rel", 1e-11)])
def test_stopping_rule_checked_with_dense_residual(tol_kind, tol):
    """The returned iterate is the FIRST one meeting the rule (Section 2.1 stopping criterion):
    checked with the dense F at the final iterate and at the iterate one update earlier."""
    pb = _newton_problem("allen_cahn", "laplacian", (), "periodic").replace(tol=tol, tol_kind=tol_kind)
    uk = _newton_input("allen_cahn")
    U, info = O.pdhg_step(pb, uk)
    Uprev, iprev = O.pdhg_step(pb.replace(max_iter=info["iterations"] - 1), uk)
    assert iprev["status"] == O.NOT_CONVERGED

    def meas(V):
        f = np.linalg.norm(dense.residual(pb, V.ravel(), uk.ravel()))
        return f / pb.dt if tol_kind == "res_abs" else f / np.linalg.norm(uk)

    assert meas(U) <= tol < meas(Uprev)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_functionalized_ch_conserves_mass_and_symbol_is_positive(bc):
    """Sixth-order functionalized CH (Section 3.3): F = U - U^k - dt Lap(...), and the sum of
    Lap(.) vanishes on both grids, so converged steps keep h^2 sum U to 1e-12; the preconditioner
    symbol (1 + dt a mu^2 (a mu + 2b - a))^2 is >= 1 with 1 exactly at the constant mode."""
    w = WL.config_fch(16)
    pb = w.problem.replace(bc=bc, tol=1e-13, tol_kind="f_rel", max_iter=20000)
    g = O.ghat(pb)
    assert g.min() == 1.0 and g[0, 0, 0] == 1.0
    U = w.u0
    m0 = O.mass(pb, U)
    for _ in range(3):
        Un, info = O.pdhg_step(pb, U)
        assert info["status"] == O.OK
        assert abs(O.mass(pb, Un) - m0) <= 1e-12 * max(1.0, abs(m0))
        U = Un
