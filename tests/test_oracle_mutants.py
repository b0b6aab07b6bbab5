"""Sensitivity of the oracle's pins, CPU only.

Each case plants one plausible mistake in the numpy oracle and checks that a committed pin
fails.  The mistakes include a dropped term, a wrong sign, index, coefficient or boundary rule,
a transposed operand, a preconditioner not squared, an extrapolation left out, and a norm or
threshold in the wrong units.  The mistake is a one-line textual change of the oracle's own
source (`oracle/rd_oracle.py`), loaded as a separate module whose functions replace the
oracle's for the duration of the case.  Each edited line must occur exactly once, so a later
change to the oracle that removes it makes the case fail loudly instead of testing nothing.
The pins are the functions of the other `tests/test_oracle_*.py` files, called unchanged: every
one passes on the unmodified oracle, and at least one of a case's pins must fail on the mutant.
The same is done for the C++ oracle (`oracle/rd_oracle_cpp.cpp`): each mutant source is compiled
with g++ into a temporary library that the ctypes binding loads in place of the built one.
"""
import inspect
import subprocess
import types

import numpy as np
import pytest

import test_oracle_3d as T3
import test_oracle_adapt as AD
import test_oracle_cpp as CPP
import test_oracle_iteration as IT
import test_oracle_operators as OPS
import test_oracle_reactions as RX
import test_oracle_stabilized as ST
from oracle import adapt, cpp_oracle, dense, rd_oracle, theory

SRC = inspect.getsource(rd_oracle)
GS = (2e-3, 1e-3, 0.04, 0.06)
SCH = (0.05, 1.0, 100.0, 0.1305, 0.7695)
O = rd_oracle

# the pins, by name: zero-argument calls of committed test functions
PINS = {
    "neumann_block_matrix": lambda: OPS.test_stencil_equals_paper_block_matrix("neumann", 4),
    "periodic_block_matrix": lambda: OPS.test_stencil_equals_paper_block_matrix("periodic", 5),
    "eigenmodes_rect_periodic": lambda: OPS.test_stencil_eigenmodes("periodic", (8, 32), (3, 2)),
    "eigenmodes_rect_neumann": lambda: OPS.test_stencil_eigenmodes("neumann", (8, 32), (3, 2)),
    "ginv_dense_ac_periodic": lambda: OPS.test_ginv_matches_dense_solve("periodic", "allen_cahn", "laplacian", ()),
    "ginv_dense_none_neumann": lambda: OPS.test_ginv_matches_dense_solve("neumann", "none", "laplacian", ()),
    "ginv_dense_ch_periodic": lambda: OPS.test_ginv_matches_dense_solve("periodic", "ch_implicit", "neg_biharmonic", ()),
    "ginv_dense_gs_neumann": lambda: OPS.test_ginv_matches_dense_solve("neumann", "gray_scott", "laplacian", GS),
    "ginv_dense_fch_periodic": lambda: OPS.test_ginv_matches_dense_solve("periodic", "fch", "functionalized", ()),
    "dense_F_fch": lambda: OPS.test_residual_matches_dense_form("periodic", "fch", "functionalized", ()),
    "adjoint_ac": lambda: OPS.test_adjoint_jacobian_by_complex_step("periodic", "allen_cahn", "laplacian", ()),
    "adjoint_ch": lambda: OPS.test_adjoint_jacobian_by_complex_step("neumann", "ch_implicit", "neg_biharmonic", ()),
    "adjoint_gs": lambda: OPS.test_adjoint_jacobian_by_complex_step("periodic", "gray_scott", "laplacian", GS),
    "adjoint_sch": lambda: OPS.test_adjoint_jacobian_by_complex_step("neumann", "schnakenberg", "laplacian", SCH),
    "adjoint_fch": lambda: OPS.test_adjoint_jacobian_by_complex_step("periodic", "fch", "functionalized", ()),
    "ac_uniform_ode": lambda: RX.test_allen_cahn_uniform_step_is_the_ode_step(0.3, O),
    "ac_mode_on_one": lambda: RX.test_allen_cahn_mode_on_a_steady_state("periodic", 2, 3, 1.0, O),
    "ch_split_mode_0": lambda: RX.test_cahn_hilliard_split_mode("periodic", 1, 2, 0.0, O),
    "ch_split_mode_045": lambda: RX.test_cahn_hilliard_split_mode("neumann", 3, 2, 0.45, O),
    "ch_implicit_mode": lambda: RX.test_cahn_hilliard_implicit_mode("periodic", 1, 2, 0.45, O),
    "gs_uniform_ode": lambda: RX.test_gray_scott_uniform_step_is_the_ode_step("periodic", 1.0, O),
    "gs_mode_per_species": lambda: RX.test_gray_scott_mode_on_the_trivial_state_decays_per_species("periodic", 3, 1, O),
    "sch_uniform_ode": lambda: RX.test_schnakenberg_uniform_step_is_the_ode_step(1 / 1000, O),
    "recurrence_unit": lambda: IT.test_single_mode_history_matches_recurrence("periodic", "laplacian", (1.0, 1.0), 1.0, "linear"),
    "recurrence_unequal": lambda: IT.test_single_mode_history_matches_recurrence("neumann", "laplacian", (0.5, 1.6), 1.0, "linear"),
    "recurrence_omega": lambda: IT.test_single_mode_history_matches_recurrence("periodic", "neg_biharmonic", (0.9, 0.9), 0.5, "linear"),
    "nilpotent": lambda: IT.test_unit_steps_are_nilpotent("neumann"),
    "stop_rule_f_rel": lambda: IT.test_stopping_rule_checked_with_dense_residual("f_rel", 1e-11),
    "stop_rule_res_abs": lambda: IT.test_stopping_rule_checked_with_dense_residual("res_abs", 1e-8),
    "newton_ac": lambda: IT.test_nonlinear_step_matches_dense_newton("allen_cahn", "laplacian", (), "neumann"),
    "stab_jacobian_ac": lambda: ST.test_stabilized_G_is_the_squared_jacobian_at_the_equilibria("periodic", "allen_cahn", "laplacian", 2.0, 1.0),
    "stab_jacobian_ch": lambda: ST.test_stabilized_G_is_the_squared_jacobian_at_the_equilibria("neumann", "ch_implicit", "neg_biharmonic", 2.0, -1.0),
    "lap3_kron": lambda: T3.test_seven_point_laplacian_is_the_kron_sum("periodic", (3, 4, 5), O),
    "ginv3_dense_neumann": lambda: T3.test_3d_ginv_matches_dense_solve("neumann", "allen_cahn", "laplacian", (), O),
}

# (name, [(old line fragment, new fragment), ...], pins of which at least one must fail)
MUTANTS = [
    ("Neumann ghost mirrored about the boundary node",
     [("idx = np.where(idx < 0, -1 - idx, idx)", "idx = np.where(idx < 0, -idx, idx)"),
      ("idx = np.where(idx >= n, 2 * n - 1 - idx, idx)", "idx = np.where(idx >= n, 2 * n - 2 - idx, idx)")],
     ["neumann_block_matrix"]),
    ("periodic shift in the wrong direction on one side",
     [("return np.roll(u, -step, axis=axis)", "return np.roll(u, -abs(step), axis=axis)")],
     ["periodic_block_matrix", "eigenmodes_rect_periodic"]),
    ("h_y taken equal to h_x",
     [("return pb.lx / pb.nx, pb.ly / pb.ny", "return pb.lx / pb.nx, pb.lx / pb.nx")],
     ["eigenmodes_rect_periodic", "eigenmodes_rect_neumann"]),
    ("y second difference divided by h_x^2",
     [("+ (_shift(u, -2, 1, pb.bc) + _shift(u, -2, -1, pb.bc) - 2 * u) / hy ** 2",
       "+ (_shift(u, -2, 1, pb.bc) + _shift(u, -2, -1, pb.bc) - 2 * u) / hx ** 2")],
     ["eigenmodes_rect_periodic"]),
    ("z second difference divided by h_y^2",
     [("- 2 * u) / spacing_z(pb) ** 2", "- 2 * u) / hy ** 2")],
     ["lap3_kron"]),
    ("Neumann eigenvalues at the periodic frequencies",
     [('d = 1.0 if pb.bc == "periodic" else 2.0', "d = 1.0")],
     ["ginv_dense_none_neumann"]),
    ("eigenvalue factor 2 for 4",
     [("mu = (4 / hx ** 2 *", "mu = (2 / hx ** 2 *")],
     ["ginv_dense_ac_periodic"]),
    ("3-D Neumann z eigenvalues at the periodic frequency",
     [("np.sin(np.pi * kz / (d * pb.nz)) ** 2", "np.sin(np.pi * kz / pb.nz) ** 2")],
     ["ginv3_dense_neumann"]),
    ("Allen-Cahn reaction with the wrong sign",
     [("f = -b * (U ** 3 - U)", "f = b * (U ** 3 - U)")],
     ["ac_uniform_ode", "ac_mode_on_one"]),
    ("Allen-Cahn W' = u^3 + u",
     [("f = -b * (U ** 3 - U)", "f = -b * (U ** 3 + U)")],
     ["ac_uniform_ode", "ac_mode_on_one"]),
    ("Cahn-Hilliard fourth-order term with the other sign reading",
     [("return U + dt * a * L(L(U)) - Uk - dt * b * L(U ** 3 - U)",
       "return U - dt * a * L(L(U)) - Uk - dt * b * L(U ** 3 - U)")],
     ["ch_implicit_mode"]),
    ("Cahn-Hilliard implicit W' = u^3",
     [("return U + dt * a * L(L(U)) - Uk - dt * b * L(U ** 3 - U)",
       "return U + dt * a * L(L(U)) - Uk - dt * b * L(U ** 3)")],
     ["ch_implicit_mode"]),
    ("convex split: explicit term with the wrong sign",
     [("- dt * b * L(U ** 3) + dt * b * L(Uk)", "- dt * b * L(U ** 3) - dt * b * L(Uk)")],
     ["ch_split_mode_0"]),
    ("convex split: U^3 taken explicitly",
     [("- dt * b * L(U ** 3) + dt * b * L(Uk)", "- dt * b * L(Uk ** 3) + dt * b * L(Uk)")],
     ["ch_split_mode_045"]),
    ("Gray-Scott: u v^2 enters the u equation with a plus sign",
     [("Fu = u - Uk[0] - dt * (Du * L(u) - u * v * v + Ff * (1 - u))",
       "Fu = u - Uk[0] - dt * (Du * L(u) + u * v * v + Ff * (1 - u))")],
     ["gs_uniform_ode"]),
    ("Gray-Scott: feed term dropped",
     [("- u * v * v + Ff * (1 - u))", "- u * v * v)")],
     ["gs_uniform_ode", "gs_mode_per_species"]),
    ("Gray-Scott: D_v diffuses u",
     [("Du * L(u)", "Dv * L(u)")],
     ["gs_mode_per_species"]),
    ("Gray-Scott: kill rate dropped from v",
     [("+ u * v * v - (Ff + k) * v)", "+ u * v * v - Ff * v)")],
     ["gs_uniform_ode", "gs_mode_per_species"]),
    ("Schnakenberg: linear decay with the wrong sign",
     [("kap * (a_s - u + u * u * v)", "kap * (a_s + u + u * u * v)")],
     ["sch_uniform_ode"]),
    ("sixth order: the printed W'' = 3u^2",
     [("return pb.a * lap(x, pb) - pb.b * (3 * U ** 2 - 1) * x + pb.a * x",
       "return pb.a * lap(x, pb) - pb.b * (3 * U ** 2) * x + pb.a * x")],
     ["dense_F_fch"]),
    ("adjoint: Allen-Cahn reaction derivative dropped",
     [("return Pt - dt * a * L(Pt) - dt * fprime * Pt", "return Pt - dt * a * L(Pt)")],
     ["adjoint_ac"]),
    ("adjoint: Cahn-Hilliard diag(W'') and Lap in the forward order",
     [("return Pt + dt * a * L(L(Pt)) - dt * b * (3 * U ** 2 - 1) * L(Pt)",
       "return Pt + dt * a * L(L(Pt)) - dt * b * L((3 * U ** 2 - 1) * Pt)")],
     ["adjoint_ch"]),
    ("adjoint: Gray-Scott coupling blocks not transposed",
     [("+ dt * (v * v + Ff) * P - dt * v * v * Q", "+ dt * (v * v + Ff) * P + 2 * dt * u * v * Q"),
      ("gv = Q - dt * Dv * L(Q) + 2 * dt * u * v * P", "gv = Q - dt * Dv * L(Q) - dt * v * v * P")],
     ["adjoint_gs"]),
    ("adjoint: Schnakenberg coupling sign",
     [("kap * (-P + 2 * u * v * (P - Q))", "kap * (-P + 2 * u * v * (P + Q))")],
     ["adjoint_sch"]),
    ("adjoint: sixth-order W''' term dropped",
     [("return Pt - dt * s + dt * b * _fch_mu(pb, U) * (6 * U) * q", "return Pt - dt * s")],
     ["adjoint_fch"]),
    ("preconditioner A_lin instead of A_lin^2",
     [("return ((1 + pb.a * dt * mu) ** 2)[None]", "return (1 + pb.a * dt * mu)[None]")],
     ["ginv_dense_ac_periodic"]),
    ("biharmonic symbol mu instead of mu^2",
     [("return ((1 + pb.a * dt * mu ** 2) ** 2)[None]", "return ((1 + pb.a * dt * mu) ** 2)[None]")],
     ["ginv_dense_ch_periodic"]),
    ("two species: D_1 for both symbols",
     [("(1 + d2 * dt * mu) ** 2", "(1 + d1 * dt * mu) ** 2")],
     ["ginv_dense_gs_neumann"]),
    ("sixth-order symbol (2b + a) for (2b - a)",
     [("(pb.a * mu + 2 * pb.b - pb.a)) ** 2)[None]", "(pb.a * mu + 2 * pb.b + pb.a)) ** 2)[None]")],
     ["ginv_dense_fch_periodic"]),
    ("stabilised Allen-Cahn symbol with the wrong sign of s",
     [("(1 + pb.b * dt * s + pb.a * dt * mu)", "(1 - pb.b * dt * s + pb.a * dt * mu)")],
     ["stab_jacobian_ac"]),
    ("stabilised Cahn-Hilliard symbol with the wrong sign of s",
     [("(1 + pb.b * s * dt * mu + pb.a * dt * mu ** 2)", "(1 - pb.b * s * dt * mu + pb.a * dt * mu ** 2)")],
     ["stab_jacobian_ch"]),
    ("periodic solve multiplies by the symbol",
     [("np.fft.fftn(W, axes=ax) / g", "np.fft.fftn(W, axes=ax) * g")],
     ["ginv_dense_ac_periodic"]),
    ("Neumann forward DCT-II not orthonormal",
     [('Wh = sfft.dctn(W, type=2, axes=ax, norm="ortho")', "Wh = sfft.dctn(W, type=2, axes=ax)")],
     ["ginv_dense_none_neumann"]),
    ("stopping norm weighted by the cell area",
     [("s = sum(np.sqrt(np.sum(W[c] * W[c])) for c in range(W.shape[0]))",
       "s = sum(np.sqrt(np.sum(W[c] * W[c]) * pb.lx * pb.ly / (pb.nx * pb.ny)) for c in range(W.shape[0]))")],
     ["stop_rule_f_rel"]),
    ("||Res|| without the 1/h_t",
     [("return s / pb.dt, pb.tol", "return s, pb.tol")],
     ["stop_rule_res_abs"]),
    ("iteration started from U = 0 instead of U^k",
     [("U = Uk.copy() if U0 is None", "U = np.zeros_like(Uk) if U0 is None")],
     ["recurrence_unit", "recurrence_unequal"]),
    ("extrapolation left out (P~ = P_{n+1})",
     [("Pt = P + (1 + pb.omega) * pb.tau_p * Y", "Pt = P + pb.tau_p * Y")],
     ["recurrence_unit", "nilpotent"]),
    ("extrapolation weight omega taken as 1",
     [("Pt = P + (1 + pb.omega) * pb.tau_p * Y", "Pt = P + 2 * pb.tau_p * Y")],
     ["recurrence_omega"]),
    ("dual step with tau_u",
     [("P = P + pb.tau_p * Y ", "P = P + pb.tau_u * Y ")],
     ["recurrence_unequal"]),
    ("primal update with P_{n+1} instead of P~",
     [("U = U - pb.tau_u * grad_F_T(pb, U, Pt)", "U = U - pb.tau_u * grad_F_T(pb, U, P)")],
     ["recurrence_unit", "nilpotent"]),
    ("primal update with the wrong sign",
     [("U = U - pb.tau_u * grad_F_T(pb, U, Pt)", "U = U + pb.tau_u * grad_F_T(pb, U, Pt)")],
     ["recurrence_unit", "newton_ac"]),
]


def _mutant_module(edits, module=rd_oracle):
    src = SRC if module is rd_oracle else inspect.getsource(module)
    for old, new in edits:
        assert src.count(old) == 1, "the line the mutant edits is not unique in %s: %r" % (module.__name__, old)
        src = src.replace(old, new)
    m = types.ModuleType("rd_oracle_mutant")
    m.__package__ = module.__package__      # the module's own relative imports
    exec(compile(src, "rd_oracle_mutant", "exec"), m.__dict__)
    return m


def _plant(monkeypatch, edits, module=rd_oracle):
    m = _mutant_module(edits, module)
    for name, obj in vars(m).items():
        if isinstance(obj, types.FunctionType) and isinstance(getattr(module, name, None), types.FunctionType):
            monkeypatch.setattr(module, name, obj)


def _fails(pin):
    try:
        with np.errstate(all="ignore"):
            pin()
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("name", sorted(PINS))
def test_pins_pass_on_the_oracle(name):
    PINS[name]()


@pytest.mark.parametrize("name,edits,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(monkeypatch, name, edits, pins):
    _plant(monkeypatch, edits)
    assert any(_fails(PINS[p]) for p in pins), "no pin caught: " + name


def test_every_pin_is_used():
    used = {p for _, _, pins in MUTANTS for p in pins}
    assert used == set(PINS), set(PINS) - used


def test_a_neutral_edit_fails_no_pin(monkeypatch):
    """Control: an edit that keeps the arithmetic (the loaded copy of the oracle itself) fails
    none of the pins, so the cases above fail for their mistakes and not for the loading."""
    _plant(monkeypatch, [("return pb.lx / pb.nx, pb.ly / pb.ny", "return (pb.lx / pb.nx), (pb.ly / pb.ny)")])
    assert rd_oracle.spacing.__module__ == "rd_oracle_mutant" or rd_oracle.spacing.__globals__["__name__"] == "rd_oracle_mutant"
    failed = [name for name, pin in PINS.items() if _fails(pin)]
    assert failed == []


# ------------------------------------------------------------------------------------------
# the adaptive step-size rule (oracle/adapt.py), the linear theory (oracle/theory.py) and the
# dense matrices the pins compare against (oracle/dense.py)
# ------------------------------------------------------------------------------------------

AUX_PINS = {
    "rule_shrink": lambda: AD.test_step_size_rule_cases(0.4, 41, 0.2),
    "rule_at_n_hi": lambda: AD.test_step_size_rule_cases(0.4, 40, 0.4),
    "rule_at_n_lo": lambda: AD.test_step_size_rule_cases(0.4, 25, 0.4),
    "rule_cap": lambda: AD.test_step_size_rule_cases(0.8, 3, 0.8),
    "no_rule_fires": AD.test_no_rule_fires_equals_fixed_steps,
    "failed_steps": AD.test_failed_steps_shrink_and_rule_holds,
    "rate": IT.test_rate_function_and_bound,
    "iteration_matrix": IT.test_random_data_follow_preconditioned_iteration_matrix,
    "eta_gamma": lambda: IT.test_eta_gamma_closed_forms(3.0),
    "recurrence": lambda: IT.test_single_mode_history_matches_recurrence("periodic", "laplacian", (0.7, 0.7), 1.0, "linear"),
    "neumann_diagonals_as_printed": OPS.test_neumann_block_diagonals_as_printed,
    "dense_periodic_block_matrix": lambda: OPS.test_stencil_equals_paper_block_matrix("periodic", 5),
    "dense_jacobian_ac": lambda: OPS.test_adjoint_jacobian_by_complex_step("periodic", "allen_cahn", "laplacian", ()),
    "dense_F_gs": lambda: OPS.test_residual_matches_dense_form("periodic", "gray_scott", "laplacian", GS),
    "dense_G_ac": lambda: OPS.test_ginv_matches_dense_solve("periodic", "allen_cahn", "laplacian", ()),
    "dense_G_ch": lambda: OPS.test_ginv_matches_dense_solve("neumann", "ch_implicit", "neg_biharmonic", ()),
}

AUX_MUTANTS = [
    (adapt, "shrink already at M = N^*", [("if m > n_hi:", "if m >= n_hi:")], ["rule_at_n_hi"]),
    (adapt, "enlarge already at M = N_*", [("if m < n_lo:", "if m <= n_lo:")], ["rule_at_n_lo"]),
    (adapt, "no cap at h_t^0", [("return up if up <= dt0 else dt", "return up")], ["rule_cap"]),
    (adapt, "shrink by 1/eta", [("return eta * dt", "return dt / eta")], ["rule_shrink"]),
    (adapt, "last step not shortened to t_end", [("h = min(dt, t_end - t)", "h = dt")], ["failed_steps"]),
    (adapt, "accepted step does not advance the state", [("U = Un\n", "U = U\n")], ["no_rule_fires", "failed_steps"]),
    (theory, "f(t) = 1 - t below 1", [("return math.sqrt(1 - t)", "return 1 - t")], ["rate"]),
    (theory, "f(t) above 1 with t^2 + t", [("return t - 1 + math.sqrt(t * t - t)", "return t - 1 + math.sqrt(t * t + t)")],
     ["rate"]),
    (theory, "iteration matrix without the extrapolation",
     [("return np.array([[1 - (1 + omega) * t, -tau_u * lam], [tau_p * lam, 1.0]])",
       "return np.array([[1 - omega * t, -tau_u * lam], [tau_p * lam, 1.0]])")], ["iteration_matrix", "rate"]),
    (theory, "eta_* bracket with kappa for 2 kappa", [("+ 2 * kappa - 0.25 / k2", "+ kappa - 0.25 / k2")], ["eta_gamma"]),
    (theory, "gamma_* with 1 for 2", [("return math.sqrt(1 - 2 / _bracket(kappa))", "return math.sqrt(1 - 1 / _bracket(kappa))")],
     ["eta_gamma"]),
    (theory, "single-mode recurrence without the extrapolation",
     [("pt = p + (1 + omega) * tau_p * y", "pt = p + tau_p * y")], ["recurrence"]),
    (dense, "Lap^N with interior diagonals in the edge blocks",
     [("L1 = _tridiag(n, [-2.0] + [-3.0] * (n - 2) + [-2.0])", "L1 = _tridiag(n, [-3.0] * n)")],
     ["neumann_diagonals_as_printed"]),
    (dense, "Lap^P without its corner entries", [("L[0, n - 1] = 1.0", "L[0, n - 1] = 0.0")],
     ["dense_periodic_block_matrix"]),
    (dense, "dense Allen-Cahn Jacobian with W'' = 3u^2 + 1",
     [("return A + np.diag(dt * b * (3 * U ** 2 - 1))", "return A + np.diag(dt * b * (3 * U ** 2 + 1))")],
     ["dense_jacobian_ac"]),
    (dense, "dense Gray-Scott u v^2 with the wrong sign",
     [("Fu = Au @ u - uk + dt * (u * v * v) - dt * Ff * (1 - u)", "Fu = Au @ u - uk - dt * (u * v * v) - dt * Ff * (1 - u)")],
     ["dense_F_gs"]),
    (dense, "dense G = A_lin instead of A_lin^2",
     [("G[c * n:(c + 1) * n, c * n:(c + 1) * n] = A @ A", "G[c * n:(c + 1) * n, c * n:(c + 1) * n] = A")],
     ["dense_G_ac"]),
    (dense, "dense Cahn-Hilliard A_lin with the other sign", [("return [I + pb.a * pb.dt * (L @ L)]", "return [I - pb.a * pb.dt * (L @ L)]")],
     ["dense_G_ch"]),
]


@pytest.mark.parametrize("name", sorted(AUX_PINS))
def test_aux_pins_pass_on_the_oracle(name):
    AUX_PINS[name]()


@pytest.mark.parametrize("module,name,edits,pins", AUX_MUTANTS, ids=[m[1] for m in AUX_MUTANTS])
def test_planted_mistake_in_the_rule_or_theory_fails_a_pin(monkeypatch, module, name, edits, pins):
    _plant(monkeypatch, edits, module)
    assert any(_fails(AUX_PINS[p]) for p in pins), "no pin caught: " + name


def test_every_aux_pin_is_used():
    used = {p for _, _, _, pins in AUX_MUTANTS for p in pins}
    assert used == set(AUX_PINS), set(AUX_PINS) - used

# ------------------------------------------------------------------------------------------
# the C++ oracle
# ------------------------------------------------------------------------------------------

CPP_SRC = open(cpp_oracle.SRC).read()
C = cpp_oracle

CPP_PINS = {
    "fft_is_the_dft": lambda: CPP.test_fft_is_the_dft(32),
    "dct_pair": lambda: CPP.test_dct_pair_is_the_orthonormal_dct2(32),
    "vs_numpy_ac_periodic": lambda: CPP.test_cpp_oracle_equals_numpy_oracle("periodic", "allen_cahn", "laplacian", (), (16, 16)),
    "vs_numpy_ac_neumann": lambda: CPP.test_cpp_oracle_equals_numpy_oracle("neumann", "allen_cahn", "laplacian", (), (16, 16)),
    "vs_numpy_split": lambda: CPP.test_cpp_oracle_equals_numpy_oracle("periodic", "ch_split", "neg_biharmonic", (), (16, 16)),
    "vs_numpy_gs": lambda: CPP.test_cpp_oracle_equals_numpy_oracle("periodic", "gray_scott", "laplacian", GS, (16, 16)),
    "vs_numpy_fch": lambda: CPP.test_cpp_oracle_equals_numpy_oracle("periodic", "fch", "functionalized", (), (16, 16)),
    "nilpotent": lambda: CPP.test_unit_steps_are_nilpotent("periodic"),
    "vs_numpy_res_abs": lambda: CPP.test_cpp_oracle_equals_numpy_oracle_with_the_res_abs_rule("periodic", "allen_cahn", "laplacian", ()),
    "ac_uniform_ode": lambda: RX.test_allen_cahn_uniform_step_is_the_ode_step(0.3, C),
    "ch_split_mode_0": lambda: RX.test_cahn_hilliard_split_mode("periodic", 1, 2, 0.0, C),
    "gs_uniform_ode": lambda: RX.test_gray_scott_uniform_step_is_the_ode_step("periodic", 1.0, C),
    "sch_uniform_ode": lambda: RX.test_schnakenberg_uniform_step_is_the_ode_step(1 / 1000, C),
    "lap3_kron": lambda: T3.test_seven_point_laplacian_is_the_kron_sum("neumann", (3, 4, 5), C),
    "ginv3_dense_gs": lambda: T3.test_3d_ginv_matches_dense_solve("periodic", "gray_scott", "laplacian", GS, C),
}

CPP_MUTANTS = [
    ("Neumann ghost one point inside", [("return j < 0 ? 0 : n - 1;", "return j < 0 ? 1 : n - 2;")],
     ["vs_numpy_ac_neumann", "lap3_kron"]),
    ("h_y from the x side length",
     [("hy2 = 1.0 / ((pb.ly / ny) * (pb.ly / ny))", "hy2 = 1.0 / ((pb.lx / ny) * (pb.lx / ny))")],
     ["vs_numpy_ac_periodic", "lap3_kron"]),
    ("z second difference weighted by h_y", [("- 2.0 * c) * hz2;", "- 2.0 * c) * hy2;")], ["lap3_kron"]),
    ("Allen-Cahn reaction with the wrong sign",
     [("const double f = -b * (U[q] * U[q] * U[q] - U[q]);", "const double f = b * (U[q] * U[q] * U[q] - U[q]);")],
     ["ac_uniform_ode"]),
    ("convex split: explicit term with the wrong sign",
     [("if (!impl) W[q] += dt * b * Lk[q];", "if (!impl) W[q] -= dt * b * Lk[q];")], ["ch_split_mode_0"]),
    ("Gray-Scott: u v^2 with a plus sign in u",
     [("- dt * (Du * Lu[q] - uvv + F * (1.0 - u[q]));", "- dt * (Du * Lu[q] + uvv + F * (1.0 - u[q]));")],
     ["gs_uniform_ode"]),
    ("Gray-Scott: kill rate dropped", [("+ uvv - (F + k) * v[q]);", "+ uvv - F * v[q]);")], ["gs_uniform_ode"]),
    ("Schnakenberg: linear decay with the wrong sign", [("kap * (as - u[q] + u2v)", "kap * (as + u[q] + u2v)")],
     ["sch_uniform_ode"]),
    ("sixth order: the printed W'' = 3u^2",
     [("o[q] = pb.a * L[q] - pb.b * (3.0 * U[q] * U[q] - 1.0) * x[q] + pb.a * x[q];",
       "o[q] = pb.a * L[q] - pb.b * (3.0 * U[q] * U[q]) * x[q] + pb.a * x[q];")],
     ["vs_numpy_fch"]),
    ("adjoint: Allen-Cahn reaction derivative dropped",
     [("g[q] = Pt[q] - dt * a * L[q] - dt * fp * Pt[q];", "g[q] = Pt[q] - dt * a * L[q];")],
     ["vs_numpy_ac_periodic"]),
    ("adjoint: Gray-Scott coupling blocks not transposed",
     [("- dt * v[q] * v[q] * Q[q];", "+ 2.0 * dt * u[q] * v[q] * Q[q];")], ["vs_numpy_gs"]),
    ("FFT: the inverse with the forward sign", [("const double ang = sgn * 2.0 * kPi * k / len;",
                                                 "const double ang = -2.0 * kPi * k / len;")], ["fft_is_the_dft"]),
    ("FFT: bit reversal left out", [("if (i < j) std::swap(x[i], x[j]);", "")], ["fft_is_the_dft"]),
    ("DCT-II: k = 0 scaled like the others",
     [("X[k] = C * (k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n));", "X[k] = C * std::sqrt(2.0 / n);")],
     ["dct_pair"]),
    ("DCT-III: Z_0 not doubled",
     [("const double s = k == 0 ? 2.0 * std::sqrt(1.0 / n) : std::sqrt(2.0 / n);",
       "const double s = k == 0 ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);")], ["dct_pair"]),
    ("Neumann eigenvalues at the periodic frequencies",
     [("d = pb.bc == BC_PERIODIC ? 1.0 : 2.0;", "d = 1.0;")], ["vs_numpy_ac_neumann"]),
    ("preconditioner A_lin instead of A_lin^2", [("g[c * n + q] = r * r;", "g[c * n + q] = r;")],
     ["nilpotent", "vs_numpy_ac_periodic"]),
    ("two species: D_1 for both symbols", [("r = 1.0 + pb.p[c] * dt * m;", "r = 1.0 + pb.p[0] * dt * m;")],
     ["ginv3_dense_gs", "vs_numpy_gs"]),
    ("periodic inverse transform not normalised",
     [("Y[q] = z[q].real() / (double)n;", "Y[q] = z[q].real();")], ["nilpotent"]),
    ("extrapolation left out",
     [("Pt[q] = P[q] + (1.0 + pb.omega) * pb.tau_p * Y[q];", "Pt[q] = P[q] + pb.tau_p * Y[q];")],
     ["nilpotent"]),
    ("||Res|| without the 1/h_t", [("*r = s / pb.dt;", "*r = s;")], ["vs_numpy_res_abs"]),
    ("adjoint: convex split with W'' = 3u^2 - 1",
     [("const double sh = pb.kind == K_CH_IMPLICIT ? 1.0 : 0.0;", "const double sh = 1.0;")], ["vs_numpy_split"]),
]


def _plant_cpp(monkeypatch, tmp_path, edits):
    src = CPP_SRC
    for old, new in edits:
        assert src.count(old) == 1, "the line the mutant edits is not unique in the C++ oracle: %r" % old
        src = src.replace(old, new)
    cpp, so = tmp_path / "rd_oracle_mutant.cpp", tmp_path / "librd_oracle_mutant.so"
    cpp.write_text(src)
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", str(so), str(cpp)],
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    assert r.returncode == 0, r.stdout.decode(errors="replace")
    monkeypatch.setattr(cpp_oracle, "LIB", str(so))
    monkeypatch.setattr(cpp_oracle, "up_to_date", lambda: True)
    monkeypatch.setattr(cpp_oracle, "_lib", None)
    cpp_oracle.set_threads(1)


@pytest.mark.parametrize("name", sorted(CPP_PINS))
def test_cpp_pins_pass_on_the_oracle(name):
    cpp_oracle.set_threads(1)
    CPP_PINS[name]()


@pytest.mark.parametrize("name,edits,pins", CPP_MUTANTS, ids=[m[0] for m in CPP_MUTANTS])
def test_planted_mistake_in_the_cpp_oracle_fails_a_pin(monkeypatch, tmp_path, name, edits, pins):
    _plant_cpp(monkeypatch, tmp_path, edits)
    assert any(_fails(CPP_PINS[p]) for p in pins), "no pin caught: " + name


def test_every_cpp_pin_is_used():
    used = {p for _, _, pins in CPP_MUTANTS for p in pins}
    assert used == set(CPP_PINS), set(CPP_PINS) - used


def test_a_neutral_edit_of_the_cpp_oracle_fails_no_pin(monkeypatch, tmp_path):
    _plant_cpp(monkeypatch, tmp_path, [("return j < 0 ? 0 : n - 1;", "return (j < 0) ? 0 : (n - 1);")])
    assert cpp_oracle.load()._name.endswith("librd_oracle_mutant.so")
    failed = [name for name, pin in CPP_PINS.items() if _fails(pin)]
    assert failed == []
