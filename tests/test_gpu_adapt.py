"""GPU: changing h_t on a live handle and the adaptive time step size of Section 2.2
("Adaptive time stepsize"), through the C ABI, against the CPU oracle."""
import dataclasses

import numpy as np
import pytest

from oracle import adapt as A, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_03945_gb300 import build
    build.build()


def _rd():
    from paper_2305_03945_gb300 import rd
    return rd


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision,loop", [("fp64", "graph"), ("fp32_dc", "graph"), ("fp32_dc", "host")])
@pytest.mark.parametrize("kind,op,p,bc", [
    ("allen_cahn", "laplacian", (), "neumann"),
    ("ch_split", "neg_biharmonic", (), "periodic"),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic"),
])
def test_set_dt_equals_a_handle_created_with_that_dt(precision, loop, kind, op, p, bc):
    """rd_pdhg_set_dt re-derives everything that depends on h_t: a step after set_dt(dt2) is bit
    for bit the step of a handle created with dt2 (same tiles, same kernels)."""
    rd = _rd()
    ch = op == "neg_biharmonic"
    dt1, dt2 = (1e-5, 3e-6) if ch else (2e-3, 5e-4)
    pb = WL.Problem(nx=64, ny=32, lx=1.0, ly=1.3, bc=bc, op=op, kind=kind, p=p, dt=dt1,
                    a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0, tau_u=0.9, tau_p=0.9, tol=1e-12,
                    tol_kind="f_rel", max_iter=3000)
    r = WL.rng(50)
    uk = (np.stack([1 - 0.5 * r.random((32, 64)), 0.25 * r.random((32, 64))]) if kind == "gray_scott"
          else r.uniform(-0.8, 0.8, pb.shape))
    outs = []
    for how in ("set", "fresh"):
        q = pb if how == "set" else dataclasses.replace(pb, dt=dt2)
        with rd.Solver(q, precision=precision, solve_loop=loop) as s:
            if how == "set":
                s.set_dt(dt2)
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = s.step(dev(uk), out)
            outs.append((host(out), info["iterations"], info["outer_rounds"]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1:] == outs[1][1:]
    U_ref, _ = O.pdhg_step(dataclasses.replace(pb, dt=dt2), uk)
    assert np.linalg.norm(outs[0][0] - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def _ac(n=32, b=50.0, dt0=0.08, max_iter=300):
    return WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc="periodic", op="laplacian", kind="allen_cahn",
                      dt=dt0, a=1.0 / b, b=b, tau_u=1.0, tau_p=1.0, tol=1e-10, tol_kind="f_rel",
                      max_iter=max_iter)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_adaptive_steps_follow_the_rule_and_match_the_oracle(precision):
    """Allen-Cahn with b h_t^0 = 4 (the first steps fail): the attempts the library logs follow the
    rule from their own iteration counts (failed -> eta h_t; the three cases after an accepted
    step; the last step shortened to t_end), the run ends at t_end, and the oracle replaying the
    accepted step sizes gives the same state.  In FP64 the iteration counts are the oracle's, so
    the whole attempt log equals the oracle's adaptive run."""
    rd = _rd()
    pb = _ac()
    u0 = WL.rng(51).uniform(-0.8, 0.8, pb.shape)
    n_hi, n_lo, eta, t_end = 40, 25, 0.5, 0.03
    u = dev(u0)
    with rd.Solver(pb, precision=precision) as s:
        log, t, st = s.solve_adaptive(u, t_end, n_hi, n_lo, eta, max_attempts=200)
        assert s.stats()  # handle still usable
    U = host(u)
    assert st == rd.RD_OK and abs(t - t_end) <= 1e-12 * t_end
    assert not log[0]["accepted"] and log[0]["status"] in (rd.RD_ERR_DIVERGED, rd.RD_ERR_NOT_CONVERGED)
    dt = pb.dt
    for e in log:
        assert e["dt"] == min(dt, t_end - e["t"])
        assert e["accepted"] == (e["status"] == rd.RD_OK)
        dt = A.next_dt(dt, e["iterations"], pb.dt, n_hi, n_lo, eta) if e["accepted"] else eta * dt
    acc = [e["dt"] for e in log if e["accepted"]]
    U_rep, infos = A.replay(pb, u0, acc)
    assert all(i["status"] == O.OK for i in infos)
    assert np.linalg.norm(U - U_rep) <= 1e-9 * np.linalg.norm(U_rep)
    if precision == "fp64":
        U_ad, log_ref, _ = A.solve_adaptive(pb, u0, t_end, n_hi, n_lo, eta, max_attempts=200)
        if [e["iterations"] for e in log if e["accepted"]] == [e["iterations"] for e in log_ref if e["accepted"]]:
            assert [e["dt"] for e in log] == [e["dt"] for e in log_ref]
        assert rel_max(U, U_ad) <= 1e-9


def test_adaptive_argument_checks_and_attempt_bound():
    """Bad parameters are refused before any work; running out of attempts returns
    RD_ERR_NOT_CONVERGED with u at the last accepted state and h_t^0 restored."""
    rd = _rd()
    pb = _ac(n=16)
    u0 = WL.rng(52).uniform(-0.8, 0.8, pb.shape)
    u = dev(u0)
    with rd.Solver(pb) as s:
        for bad in [dict(t_end=0.0, n_hi=40, n_lo=25, eta=0.5), dict(t_end=0.03, n_hi=40, n_lo=25, eta=1.0),
                    dict(t_end=0.03, n_hi=20, n_lo=25, eta=0.5)]:
            with pytest.raises(rd.RDError):
                s.solve_adaptive(u, **bad)
        log, t, st = s.solve_adaptive(u, 0.1, 40, 25, 0.5, max_attempts=3, allow=(rd.RD_ERR_NOT_CONVERGED,))
        assert st == rd.RD_ERR_NOT_CONVERGED and len(log) == 3 and t == 0.0
        assert np.array_equal(host(u), u0)      # every attempt failed: the state is untouched
        # h_t^0 is back: a plain step is the step of the original h_t
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(u0), out, allow=(rd.RD_OK, rd.RD_ERR_DIVERGED, rd.RD_ERR_NOT_CONVERGED))
        assert info["status"] == log[0]["status"] and info["iterations"] == log[0]["iterations"]
