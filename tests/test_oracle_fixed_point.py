"""Pins of the oracle's second solver of the implicit Cahn-Hilliard step (oracle/fixed_point.py),
CPU only: its root satisfies F(U) = 0 of the PDHG oracle and equals the PDHG oracle's step."""
import dataclasses

import numpy as np

from oracle import fixed_point as FP, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL


def test_fixed_point_step_is_the_pdhg_step():
    """Seven-circle data on 32^2 and a random field on 16x32: the fixed-point root and the PDHG
    root agree to 1e-11 (the PDHG stop is ||F|| <= 1e-13 ||U^k||) and the fixed point makes
    ||F|| tiny."""
    w = WL.config_seven_circles(32)
    cases = [(w.problem, w.u0)]
    pb = WL.Problem(nx=32, ny=16, lx=1.0, ly=0.5, bc="periodic", op="neg_biharmonic", kind="ch_implicit",
                    a=1e-3, b=1.0, dt=1e-4, tau_u=1.0, tau_p=1.0, tol=1e-13, tol_kind="f_rel")
    cases.append((pb, WL.rng(60).uniform(-0.5, 0.5, pb.shape)))
    for pb, u0 in cases:
        U, its = FP.ch_implicit_step(pb, u0)
        Up, info = O.pdhg_step(dataclasses.replace(pb, tol=1e-13, tol_kind="f_rel", max_iter=20000), u0)
        assert info["status"] == O.OK
        assert np.max(np.abs(U - Up)) <= 1e-11 * np.max(np.abs(Up))
        assert np.linalg.norm(O.residual(pb, U, u0)) <= 1e-12 * np.linalg.norm(u0)


def test_sign_change_detection():
    """The sign-change bookkeeping on a short run: a point that starts positive inside the
    smallest circle (Table 1, i = 3, r = pi/15) and a point that never changes."""
    w = WL.config_seven_circles(32)
    pb = dataclasses.replace(w.problem, dt=0.05)
    U = np.asarray(w.u0)
    steps = FP.sign_change_steps(pb, U, [(20, 8), (0, 0)], 40)
    assert steps[1] is None
    if steps[0] is not None:
        V = U
        for _ in range(steps[0] - 1):
            V, _ = FP.ch_implicit_step(pb, V)
        assert np.sign(V[0, 20, 8]) == np.sign(U[0, 20, 8])
        V, _ = FP.ch_implicit_step(pb, V)
        assert np.sign(V[0, 20, 8]) != np.sign(U[0, 20, 8])
