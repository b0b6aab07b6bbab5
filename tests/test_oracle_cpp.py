"""Pins of the plain C++ FP64 oracle (oracle/rd_oracle_cpp.cpp), CPU only.

Its transforms are checked against the brute-force DFT / DCT-II definitions; the whole method
against the numpy oracle (an independent restatement with library FFT / DCT) on every equation
kind, both boundary conditions and ragged grids, iteration counts included; and directly against
closed forms the paper and the mathematics fix (the nilpotent two-iteration solve of Appendix A,
the single-mode decay rate, dense Newton).
"""
import math

import numpy as np
import pytest

from oracle import cpp_oracle as C, dense as D, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL


@pytest.fixture(scope="module", autouse=True)
def _one_thread():
    """Tiny grids: one thread (OpenMP start-up per loop would dominate)."""
    C.set_threads(1)
    yield
    C.set_threads(0)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32, 64])
def test_fft_is_the_dft(n):
    r = WL.rng(n)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    jk = np.outer(np.arange(n), np.arange(n)) % n          # exact phases: exp(-2 pi i (jk mod n) / n)
    F = np.exp(-2j * np.pi * jk / n)
    scale = np.sum(np.abs(x))
    assert np.max(np.abs(C.fft(x) - F @ x)) <= 1e-14 * scale
    assert np.max(np.abs(C.fft(x, inverse=True) - F.conj() @ x)) <= 1e-14 * scale


@pytest.mark.parametrize("n", [1, 2, 4, 8, 32, 64])
def test_dct_pair_is_the_orthonormal_dct2(n):
    x = WL.rng(n + 100).standard_normal(n)
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    M = np.cos(np.pi * k * (2 * j + 1) / (2 * n)) * np.where(k == 0, math.sqrt(1 / n), math.sqrt(2 / n))
    assert np.allclose(M @ M.T, np.eye(n), atol=1e-14)      # the basis is orthonormal
    assert np.max(np.abs(C.dct2(x) - M @ x)) <= 1e-14 * np.sum(np.abs(x))
    assert np.max(np.abs(C.dct3(M @ x) - x)) <= 1e-14 * np.sum(np.abs(x))


KINDS = [
    ("none", "laplacian", ()),
    ("none", "neg_biharmonic", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("ch_split", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
    ("fch", "functionalized", ()),
]


def _pb(kind, op, p, bc, ny, nx):
    ch = op != "laplacian"
    pb = WL.Problem(nx=nx, ny=ny, lx=1.0, ly=1.3, bc=bc, op=op, kind=kind, p=p, dt=1e-5 if ch else 2e-3,
                    a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0, tau_u=0.9, tau_p=0.9, tol=1e-12,
                    tol_kind="f_rel", max_iter=3000)
    if kind == "fch":
        pb = pb.replace(a=0.18 ** 2, b=1.0, dt=1e-6, tau_u=0.58, tau_p=0.58)
    return pb


def _state(pb, r):
    if pb.kind == "schnakenberg":
        return np.stack([np.full((pb.ny, pb.nx), 0.9), np.full((pb.ny, pb.nx), 0.95)]) * (1 + 0.05 * r.uniform(-1, 1, pb.shape))
    U = r.uniform(-0.8, 0.8, pb.shape)
    return np.abs(U) if pb.kind == "gray_scott" else U


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", KINDS)
@pytest.mark.parametrize("shape", [(2, 2), (4, 8), (16, 16), (32, 64), (64, 16)])
def test_cpp_oracle_equals_numpy_oracle(bc, kind, op, p, shape):
    pb = _pb(kind, op, p, bc, *shape)
    r = WL.rng(shape[0] * 1000 + shape[1])
    U, Uk, W = _state(pb, r), _state(pb, r), r.standard_normal(pb.shape)
    assert _rel(C.residual(pb, U, Uk), O.residual(pb, U, Uk)) <= 1e-14
    assert _rel(C.grad_F_T(pb, U, W), O.grad_F_T(pb, U, W)) <= 1e-14
    assert _rel(C.ghat(pb), O.ghat(pb)) <= 1e-14
    assert _rel(C.apply_ginv(pb, W), O.apply_ginv(pb, W)) <= 1e-13
    Ua, ia = O.pdhg_step(pb, Uk, history=True)
    Ub, ib = C.pdhg_step(pb, Uk, history=True)
    assert (ia["status"], ia["iterations"]) == (ib["status"], ib["iterations"])
    assert np.max(np.abs(ia["history"] - ib["history"])) <= 1e-11 * ia["history"][0]
    assert _rel(Ub, Ua) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", KINDS)
def test_cpp_oracle_equals_numpy_oracle_with_the_res_abs_rule(bc, kind, op, p):
    """The paper's stopping rule ||Res|| = ||F|| / h_t <= delta (Section 2.1), with delta set to
    stop near ||F|| = 1e-11: the same statuses, iteration counts, measures and results."""
    pb = _pb(kind, op, p, bc, 16, 16)
    pb = pb.replace(tol_kind="res_abs", tol=1e-11 / pb.dt)
    r = WL.rng(77)
    Uk = _state(pb, r)
    Ua, ia = O.pdhg_step(pb, Uk, history=True)
    Ub, ib = C.pdhg_step(pb, Uk, history=True)
    assert ia["status"] == O.OK
    assert (ia["status"], ia["iterations"]) == (ib["status"], ib["iterations"])
    assert np.max(np.abs(ia["history"] - ib["history"])) <= 1e-11 * ia["history"][0]
    assert _rel(Ub, Ua) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_unit_steps_are_nilpotent(bc):
    """Appendix A: reaction off, G = A^2, tau_u = tau_p = omega = 1 -- the per-mode iteration
    matrix is nilpotent, so the second iterate is the exact implicit step."""
    pb = WL.Problem(nx=16, ny=8, lx=1.0, ly=0.5, bc=bc, op="laplacian", kind="none", a=0.3, dt=0.01,
                    tau_u=1.0, tau_p=1.0, tol=1e-13, tol_kind="f_rel")
    uk = WL.rng(9).standard_normal(pb.shape)
    U, info = C.pdhg_step(pb, uk)
    assert info["status"] == C.OK and info["iterations"] == 2
    assert np.linalg.norm(C.residual(pb, U, uk)) <= 1e-13 * np.linalg.norm(uk)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_single_mode_decays_at_closed_form_rate(bc):
    """Reaction off: one eigenmode decays per implicit step by exactly 1 / (1 + dt a mu)."""
    pb = WL.Problem(nx=32, ny=32, lx=1.0, ly=1.0, bc=bc, op="laplacian", kind="none", a=0.05, dt=0.01,
                    tau_u=1.0, tau_p=1.0, tol=1e-14, tol_kind="f_rel")
    kx, ky = 3, 2
    d = 1 if bc == "periodic" else 2
    mu = 4 * 32 ** 2 * (math.sin(math.pi * kx / (d * 32)) ** 2 + math.sin(math.pi * ky / (d * 32)) ** 2)
    u0 = WL.cosine_mode(pb, kx, ky) if bc == "neumann" else WL.cosine_mode(pb, kx, ky)
    U, infos = C.solve(pb, u0, 20)
    assert all(i["status"] == C.OK for i in infos)
    assert np.max(np.abs(U - u0 * (1 + pb.dt * pb.a * mu) ** -20)) <= 1e-12


@pytest.mark.parametrize("kind,op,p,bc", [
    ("allen_cahn", "laplacian", (), "periodic"),
    ("ch_split", "neg_biharmonic", (), "neumann"),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic"),
])
def test_nonlinear_step_matches_dense_newton(kind, op, p, bc):
    """16 x 16: the PDHG step equals dense Newton on the paper's block matrices to 1e-10."""
    ch = op == "neg_biharmonic"
    pb = WL.Problem(nx=16, ny=16, lx=1.0, ly=1.0, bc=bc, op=op, kind=kind, p=p, dt=1e-5 if ch else 2e-3,
                    a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0, tau_u=0.9, tau_p=0.9, tol=1e-13,
                    tol_kind="f_rel", max_iter=20000)
    r = WL.rng(33)
    uk = _state(pb, r)
    U, info = C.pdhg_step(pb, uk)
    assert info["status"] == C.OK
    assert _rel(U, D.newton(pb, uk)) <= 1e-10


def test_thread_count_does_not_change_results():
    w = WL.config_allen_cahn_neumann(128, 1, seed=5)
    outs = []
    for t in (1, 3):
        C.set_threads(t)
        outs.append(C.pdhg_step(w.problem, w.u0))
    C.set_threads(1)
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_fixed_iteration_step_of_the_roofline_sweep():
    """The roofline sweep's step form (threshold 0, max_iter = m, Section 2.1's loop with a
    stopping rule that never holds): both oracles take exactly m updates, report not converged
    and return the same U_m; U_m moves toward the step's solution as m grows."""
    w = WL.config_allen_cahn_periodic_8192(n=32, fixed_iters=7)
    pb = w.problem
    U_n, info_n = O.pdhg_step(pb, w.u0)
    U_c, info_c = C.pdhg_step(pb, w.u0)
    assert info_n["status"] == O.NOT_CONVERGED and info_n["iterations"] == 7
    assert info_c["status"] == C.NOT_CONVERGED and info_c["iterations"] == 7
    assert np.max(np.abs(U_n - U_c)) <= 1e-12 * np.max(np.abs(U_n))
    U_ref, info_ref = O.pdhg_step(pb.replace(tol=1e-12, tol_kind="f_rel", max_iter=10000), w.u0)
    assert info_ref["status"] == O.OK
    U_3, _ = O.pdhg_step(pb.replace(max_iter=3), w.u0)
    assert np.linalg.norm(U_n - U_ref) < np.linalg.norm(U_3 - U_ref)


def test_non_power_of_two_sides_refused():
    pb = _pb("allen_cahn", "laplacian", (), "periodic", 16, 16).replace(nx=12)
    with pytest.raises(ValueError, match="power-of-two"):
        C.pdhg_step(pb, np.zeros(pb.shape))
