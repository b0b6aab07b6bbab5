"""Degenerate inputs on the GPU through the C ABI: a step that starts at a steady state and a
solve of no steps.

At a uniform steady state (Allen-Cahn u = +-1, Cahn-Hilliard any constant, the linear equations
any constant, Gray-Scott (u, v) = (1, 0)) every stencil of a constant field is exactly 0 and so is
the reaction term, so F(U^k) = 0 holds exactly in floating point: the stopping rule is met before
the first update (Section 2.1, the stop test applied to U_0 = U^k).  Every path must then report
0 iterations and return U^k bit for bit, as the CPU oracles do: FP64 on both loops, defect
correction on the band sweeps and on the one-launch small solve, 3-D grids, 2-D grids with long
lines, and batched requests next to one that iterates."""
import time

import numpy as np
import pytest

from oracle import rd_oracle as O
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


GS_P = (2e-3, 1e-3, 0.04, 0.06)
# (kind, operator, parameters, the constant state)
STEADY = [
    ("allen_cahn", "laplacian", (), 1.0),
    ("allen_cahn", "laplacian", (), -1.0),
    ("ch_implicit", "neg_biharmonic", (), 0.3),
    ("ch_split", "neg_biharmonic", (), -0.7),
    ("none", "laplacian", (), 0.0),
    ("none", "neg_biharmonic", (), 0.5),
    ("gray_scott", "laplacian", GS_P, None),
]
SCALAR = [c for c in STEADY if c[0] != "gray_scott"]


def _pb(kind, op, p, bc, ny, nx, nz=1, **kw):
    ch = op == "neg_biharmonic"
    base = dict(nx=nx, ny=ny, nz=nz, lx=1.7, ly=1.3, lz=0.9, bc=bc, op=op, kind=kind,
                dt=1.0 if kind == "gray_scott" else (1e-5 if ch else 2e-3), a=4e-4 if ch else 0.05,
                b=1.0 if ch else 20.0, tau_u=0.9, tau_p=0.9, tol=1e-11, tol_kind="f_rel", max_iter=2000)
    if p:
        base["p"] = p
    base.update(kw)
    return WL.Problem(**base)


def _state(pb, value):
    if value is None:  # Gray-Scott (u, v) = (1, 0)
        u = np.zeros(pb.shape)
        u[0] = 1.0
        return u
    return np.full(pb.shape, value)


def _assert_fixed_point_step(pb, uk, precision="fp64", **opts):
    rd = _rd()
    U_ref, info_ref = O.pdhg_step(pb, uk)
    assert info_ref["status"] == O.OK and info_ref["iterations"] == 0
    assert np.array_equal(U_ref, uk)
    with rd.Solver(pb, precision=precision, **opts) as s:
        out = torch.full(pb.shape, 7.0, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0 and info["iterations"] == 0, info
    assert np.array_equal(U, uk)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p,value", STEADY)
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_fp64_step_from_a_steady_state(bc, kind, op, p, value, loop):
    pb = _pb(kind, op, p, bc, 16, 32)
    _assert_fixed_point_step(pb, _state(pb, value), solve_loop=loop)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p,value", STEADY)
@pytest.mark.parametrize("shape,small", [((16, 32), 1), ((16, 32), 0), ((128, 256), 0)])
def test_defect_correction_step_from_a_steady_state(bc, kind, op, p, value, shape, small):
    pb = _pb(kind, op, p, bc, *shape)
    _assert_fixed_point_step(pb, _state(pb, value), precision="fp32_dc", small_solve=small)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p,value", SCALAR)
@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_3d_step_from_a_steady_state(bc, kind, op, p, value, precision):
    pb = _pb(kind, op, p, bc, 8, 16, nz=4)
    _assert_fixed_point_step(pb, _state(pb, value), precision=precision)


@pytest.mark.parametrize("kind,op,p,value", SCALAR)
@pytest.mark.parametrize("precision,shape", [("fp64", (4, 8192)), ("fp32_dc", (4096, 16))])
def test_long_line_step_from_a_steady_state(kind, op, p, value, precision, shape):
    """Side lengths in proportion to the points (h about 0.02).  The line kernels' 25-point
    Lap^2 sums each axis' weights 1, -4, 6, -4, 1 of the point values, which for a constant c
    cancels only to about eps |c|, then scales by 1/h^4: on [0,1.7) x [0,1.3) with 8192 points
    (h = 2e-4) F(U^k) of a constant Cahn-Hilliard state is about 1e-9 per point, above the
    1e-11 relative threshold, and the step takes a few hundred iterations to converge (measured;
    the oracle's nested Laplacians cancel exactly)."""
    rd = _rd()
    ny, nx = shape
    pb = _pb(kind, op, p, "periodic", ny, nx, lx=1.7 * nx / 64, ly=1.3 * ny / 64)
    with rd.Solver(pb, precision=precision) as s:
        assert s.stats()["line_kernels"] == 1
    _assert_fixed_point_step(pb, _state(pb, value), precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_solve_of_no_steps_leaves_the_state(precision):
    rd = _rd()
    pb = _pb("allen_cahn", "laplacian", (), "neumann", 32, 32)
    uk = WL.rng(31).uniform(-0.9, 0.9, pb.shape)
    u = dev(uk)
    with rd.Solver(pb, precision=precision) as s:
        infos, status = s.solve(u, 0)
        uh = uk.copy()
        infos_h, status_h = s.solve_host(uh, 0)
    assert status == 0 and infos == [] and status_h == 0 and infos_h == []
    assert np.array_equal(host(u), uk) and np.array_equal(uh, uk)


def test_batched_steady_states_next_to_an_iterating_request():
    rd = _rd()
    reqs = []
    for kind, op, p, value in [STEADY[0], STEADY[2], STEADY[3], STEADY[6]]:
        pb = _pb(kind, op, p, "periodic", 32, 64)
        reqs.append((pb, _state(pb, value)))
    pb = _pb("allen_cahn", "laplacian", (), "neumann", 64, 64)
    reqs.append((pb, WL.rng(32).uniform(-0.9, 0.9, pb.shape)))
    results, outs = {}, {}
    with rd.Batch(1 << 30, 8) as b:
        ids = []
        for k, (pb, u0) in enumerate(reqs):
            rid, out = b.submit(pb, u0, 2, tag=k)
            ids.append(rid)
            outs[rid] = out
        t0 = time.time()
        while len(results) < len(ids) and time.time() - t0 < 120:
            for r in b.poll(timeout=1.0):
                results[r["id"]] = r
    assert len(results) == len(reqs)
    for k, (rid, (pb, u0)) in enumerate(zip(ids, reqs)):
        r = results[rid]
        assert r["status"] == 0 and r["steps"] == 2, r
        if k < 4:
            assert r["iterations"] == 0, r
            assert np.array_equal(outs[rid], u0)
        else:
            assert r["iterations"] > 0
            U_ref, _ = O.solve(pb, u0, 2)
            assert np.linalg.norm(outs[rid] - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
