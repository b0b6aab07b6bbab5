"""Pins of the oracle's adaptive time step size (Section 2.2, "Adaptive time stepsize"), CPU only.

The rule is host logic on the PDHG iteration count; it is pinned by the paper's three cases
worked by hand, by its reduction to Algorithm 1's fixed-step loop when no case fires, and by an
Allen-Cahn run whose first step sizes make PDHG fail, so that every branch (failed attempt,
shrink, keep, enlarge, the h_t^0 cap and the shortened last step) is taken."""
import numpy as np
import pytest

from oracle import adapt as A, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL


@pytest.mark.parametrize("dt,m,expect", [
    (0.4, 41, 0.2),      # M > N^*: shrink by eta
    (0.4, 40, 0.4),      # M = N^*: unchanged
    (0.4, 25, 0.4),      # M = N_*: unchanged
    (0.4, 24, 0.8),      # M < N_*: enlarge by 1/eta (0.8 <= h_t^0 = 1)
    (0.8, 3, 0.8),       # M < N_*, but 0.8 / 0.5 = 1.6 > h_t^0: unchanged
    (1.0, 0, 1.0),       # at the cap
])
def test_step_size_rule_cases(dt, m, expect):
    """The three cases of the rule with N^* = 40, N_* = 25, eta = 1/2, h_t^0 = 1."""
    assert A.next_dt(dt, m, 1.0, 40, 25, 0.5) == expect


def _ac(n=16, b=50.0, dt0=0.08, max_iter=300):
    return WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="periodic", op="laplacian", kind="allen_cahn",
                      dt=dt0, a=1.0 / b, b=b, tau_u=1.0, tau_p=1.0, tol=1e-10, tol_kind="f_rel",
                      max_iter=max_iter)


def test_no_rule_fires_equals_fixed_steps():
    """With N_* = 0 and N^* above max_iter no case changes h_t: the run is Algorithm 1's loop of
    t_end / h_t^0 fixed steps, bit for bit."""
    pb = _ac(b=10.0, dt0=2e-3)
    u0 = WL.rng(40).uniform(-0.8, 0.8, pb.shape)
    U, log, t = A.solve_adaptive(pb, u0, 6 * pb.dt, n_hi=10 ** 6, n_lo=0, eta=0.5)
    U_ref, infos = O.solve(pb, u0, 6)
    assert [e["accepted"] for e in log] == [True] * 6
    assert [e["iterations"] for e in log] == [i["iterations"] for i in infos]
    assert np.array_equal(U, U_ref)
    assert abs(t - 6 * pb.dt) <= 1e-15


def test_failed_steps_shrink_and_rule_holds():
    """Allen-Cahn with b h_t^0 = 4: the implicit step is not monotone and PDHG fails, so the first
    attempts are rejected and h_t halves until a step converges.  Afterwards every accepted step
    meets the stopping rule, each h_t follows from the previous one by the three cases, no h_t
    exceeds h_t^0, the run ends exactly at t_end, and replaying the accepted step sizes as fixed
    steps gives the same state."""
    pb = _ac()
    u0 = WL.rng(41).uniform(-0.8, 0.8, pb.shape)
    n_hi, n_lo, eta, t_end = 40, 25, 0.5, 0.03
    U, log, t = A.solve_adaptive(pb, u0, t_end, n_hi, n_lo, eta)
    assert not log[0]["accepted"] and log[0]["status"] in (O.DIVERGED, O.NOT_CONVERGED)
    acc = [e for e in log if e["accepted"]]
    assert acc and abs(t - t_end) <= 1e-12 * t_end
    assert abs(sum(e["dt"] for e in acc) - t_end) <= 1e-12 * t_end
    # the rule, attempt by attempt (a step is shortened where it would pass t_end)
    dt = pb.dt
    kinds = set()
    for e in log:
        assert e["dt"] == min(dt, t_end - e["t"])
        if not e["accepted"]:
            dt, kind = eta * dt, "failed"
        else:
            nd = A.next_dt(dt, e["iterations"], pb.dt, n_hi, n_lo, eta)
            kind = "shrink" if nd < dt else ("enlarge" if nd > dt else "keep")
            dt = nd
        kinds.add(kind)
    assert kinds == {"failed", "shrink", "keep", "enlarge"}
    # every accepted step converged: replaying its size from the same state reproduces it
    U_rep, infos = A.replay(pb, u0, [e["dt"] for e in acc])
    assert all(i["status"] == O.OK for i in infos)
    assert [i["iterations"] for i in infos] == [e["iterations"] for e in acc]
    assert np.array_equal(U_rep, U)
