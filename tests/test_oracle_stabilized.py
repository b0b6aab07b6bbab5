"""Pins of the stabilised preconditioner (precond 'stabilized'): the square of F's Jacobian with
its nonlinear factor replaced by a constant s, Section 3.3's construction of G, applied to any
scalar reaction.  At the equilibria u = +-1 the factor is that constant (W''(+-1) = 2 for
Allen-Cahn and implicit Cahn-Hilliard, 3 U^2 = 3 for the convex split), so there G must be the
square of the exact Jacobian, which oracle/dense.py assembles independently from the residual's
derivative.  The fixed point of the iteration does not depend on G (dense Newton), and near the
equilibria the stabilised G keeps PDHG convergent where G = A_lin^2 diverges."""
import numpy as np
import pytest

from oracle import cpp_oracle as C, dense as D, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL

CASES = [("allen_cahn", "laplacian", 2.0), ("ch_implicit", "neg_biharmonic", 2.0), ("ch_split", "neg_biharmonic", 3.0)]


@pytest.fixture(scope="module", autouse=True)
def _one_thread():
    C.set_threads(1)
    yield
    C.set_threads(0)


def _pb(kind, op, bc, n, s, **kw):
    lap = op == "laplacian"
    base = dict(nx=n, ny=n, lx=1.3, ly=1.3, bc=bc, op=op, kind=kind, dt=2e-3 if lap else 1e-4,
                a=0.05 if lap else 1e-3, b=20.0 if lap else 1.0, precond="stabilized", shift=s)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
@pytest.mark.parametrize("value", [1.0, -1.0])
def test_stabilized_G_is_the_squared_jacobian_at_the_equilibria(bc, kind, op, s, value):
    pb = _pb(kind, op, bc, 8, s)
    J = D.jacobian(pb, np.full(pb.nx * pb.ny, value))
    x = WL.rng(3).standard_normal(pb.shape)
    GX = (J @ (J @ x.ravel())).reshape(pb.shape)
    assert np.max(np.abs(O.apply_ginv(pb, GX) - x)) <= 1e-12
    assert np.max(np.abs(C.apply_ginv(pb, GX) - x)) <= 1e-12


def test_stabilized_sixth_order_with_s_2_is_the_paper_G():
    w = WL.config_fch(16)
    pb = w.problem
    g_lin = O.ghat(pb)
    g_stab = O.ghat(pb.replace(precond="stabilized", shift=2.0))
    assert np.max(np.abs(g_stab - g_lin)) <= 1e-12 * np.max(g_lin)
    g_c = C.ghat(pb.replace(precond="stabilized", shift=2.0))
    assert np.max(np.abs(g_c - g_lin)) <= 1e-12 * np.max(g_lin)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
def test_stabilized_step_reaches_the_dense_newton_solution(bc, kind, op, s):
    pb = _pb(kind, op, bc, 8, s, tau_u=0.9, tau_p=0.9, tol=1e-13, tol_kind="f_rel", max_iter=5000)
    uk = WL.rng(5).uniform(-0.9, 0.9, pb.shape)
    U, info = O.pdhg_step(pb, uk)
    assert info["status"] == O.OK
    Un = D.newton(pb, uk).reshape(pb.shape)
    assert np.max(np.abs(U - Un)) <= 1e-10
    Uc, info_c = C.pdhg_step(pb, uk)
    assert info_c["iterations"] == info["iterations"]
    assert np.max(np.abs(Uc - U)) <= 1e-12


def _near_equilibrium(n):
    x = np.arange(n) * 2 * np.pi / n
    return np.tanh(3 * np.sin(x)[None, :] * np.cos(x)[:, None])[None]


@pytest.mark.parametrize("kind,op,kw", [
    ("allen_cahn", "laplacian", dict(a=0.1, b=10.0, dt=0.05)),
    ("ch_implicit", "neg_biharmonic", dict(a=4e-4, b=1.0, dt=1e-4, lx=1.0, ly=1.0)),
])
def test_stabilized_keeps_the_iteration_convergent_near_the_equilibria(kind, op, kw):
    """A state near +-1 with a stiff reaction term: with G = A_lin^2 the iteration diverges,
    with the stabilised G (s = W''(+-1) = 2) it converges."""
    n = 32
    base = dict(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc="periodic", op=op, kind=kind, tau_u=1.0,
                tau_p=1.0, tol=1e-10, tol_kind="f_rel", shift=2.0)
    base.update(kw)
    u0 = _near_equilibrium(n)
    _, info_lin = O.pdhg_step(WL.Problem(precond="linear", **base), u0)
    U, info = O.pdhg_step(WL.Problem(precond="stabilized", **base), u0)
    assert info_lin["status"] == O.DIVERGED
    assert info["status"] == O.OK
    r, thr = O.measure(WL.Problem(precond="stabilized", **base), O.residual(WL.Problem(**base), U, u0), u0)
    assert r <= thr


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
def test_stabilized_with_s_0_is_the_linear_G(bc, kind, op, s):
    """With the nonlinear factor set to 0 the Jacobian is the linear part's: G = A_lin^2."""
    pb = _pb(kind, op, bc, 16, 0.0)
    lin = pb.replace(precond="linear", shift=0.0)
    for M in (O, C):
        g0, gl = M.ghat(pb), M.ghat(lin)
        assert np.max(np.abs(g0 - gl)) <= 1e-14 * np.max(gl)
    uk = WL.rng(6).uniform(-0.9, 0.9, pb.shape)
    p0 = pb.replace(tau_u=0.9, tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=3000)
    U0, i0 = O.pdhg_step(p0, uk)
    Ul, il = O.pdhg_step(p0.replace(precond="linear"), uk)
    assert i0["iterations"] == il["iterations"]
    assert np.max(np.abs(U0 - Ul)) <= 1e-14 * np.max(np.abs(Ul))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
@pytest.mark.parametrize("value", [1.0, -1.0])
def test_stabilized_G_on_3d_grids_is_the_squared_jacobian_at_the_equilibria(bc, kind, op, s, value):
    """The same construction with a third axis (the Kronecker-sum Laplacian of the dense module)."""
    pb = _pb(kind, op, bc, 4, s, nz=4, ny=4, nx=8, lx=1.0, ly=0.8, lz=1.3)
    J = D.jacobian(pb, np.full(pb.nx * pb.ny * pb.nz, value))
    x = WL.rng(4).standard_normal(pb.shape)
    GX = (J @ (J @ x.ravel())).reshape(pb.shape)
    assert np.max(np.abs(O.apply_ginv(pb, GX) - x)) <= 1e-12
    assert np.max(np.abs(C.apply_ginv(pb, GX) - x)) <= 1e-12
