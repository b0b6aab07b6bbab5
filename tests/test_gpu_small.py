"""The one-launch inner solve of FP32 defect correction (rd_opts.small_solve: every array of a
small 2-D grid's inner PDHG solve in shared memory -- of one block below 16 points a side, of a
cluster of eight blocks up to 16 K points -- one launch per inner solve) against the CPU oracle
and against the multi-kernel sweeps, through the C ABI.  Tolerance as for
every defect-correction step: relative L2 error <= 1e-9 per step."""
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


KINDS = [
    ("none", "laplacian", ()),
    ("none", "neg_biharmonic", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("ch_split", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
]
SHAPES = [(2, 2), (4, 8), (8, 32), (16, 16), (32, 64), (64, 64), (128, 128)]


def _pb(kind, op, p, bc, ny, nx):
    ch = op == "neg_biharmonic"
    return WL.Problem(nx=nx, ny=ny, lx=1.0, ly=1.3, bc=bc, op=op, kind=kind, p=p,
                      dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                      tau_u=0.9, tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=3000)


def _state(pb, seed):
    r = WL.rng(seed)
    if pb.kind == "gray_scott":
        return np.stack([1 - 0.5 * r.random((pb.ny, pb.nx)), 0.25 * r.random((pb.ny, pb.nx))])
    if pb.kind == "schnakenberg":
        return 0.9 + 0.1 * r.random(pb.shape)
    return r.uniform(-0.8, 0.8, pb.shape)


def _step(pb, uk, **opts):
    rd = _rd()
    with rd.Solver(pb, precision="fp32_dc", **opts) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        st = s.stats()
        return host(out), info, st


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", KINDS)
@pytest.mark.parametrize("shape", SHAPES)
def test_small_solve_step_matches_oracle(bc, kind, op, p, shape):
    pb = _pb(kind, op, p, bc, *shape)
    uk = _state(pb, 4)
    U, info, st = _step(pb, uk)
    # one block below 16 points a side (up to 4 K points), a cluster of eight blocks from 16 x 16
    # up to 16 K points, else the multi-kernel sweeps
    npts = pb.ncomp * pb.nx * pb.ny
    want = (2 if npts <= 16384 else 0) if min(shape) >= 16 else (1 if npts <= 4096 else 0)
    assert st["small_solve"] == want
    assert info["status"] == 0, info
    U_ref, _ = O.pdhg_step(pb, uk)
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("shape", [(64, 128), (128, 64)])
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_small_solve_equals_multi_kernel_sweeps(bc, shape, loop):
    """The largest grids the one-block solve takes, both loops: the same step as the band /
    column kernels (small_solve = 0) to the step tolerance, and both against the oracle."""
    pb = _pb("allen_cahn", "laplacian", (), bc, *shape)
    uk = _state(pb, 5)
    U1, i1, s1 = _step(pb, uk, solve_loop=loop)
    U0, i0, s0 = _step(pb, uk, solve_loop=loop, small_solve=0)
    assert s1["small_solve"] == 2 and s0["small_solve"] == 0
    U_ref, _ = O.pdhg_step(pb, uk)
    for U in (U0, U1):
        assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_small_solve_not_used_beyond_shared_memory():
    pb = _pb("allen_cahn", "laplacian", (), "periodic", 256, 256)
    U, info, st = _step(pb, _state(pb, 6))
    assert st["small_solve"] == 0 and info["status"] == 0


def test_allen_cahn_64_periodic_twenty_steps_small_solve():
    """The 64^2 periodic Allen-Cahn configuration (Section 3.1 physics) in FP32 + FP64 defect
    correction through the one-block solve: 20 steps within 1e-9 of the oracle's FP64 run."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic()
    U_ref, _ = O.solve(w.problem, w.u0, w.nsteps)
    u = dev(w.u0)
    with rd.Solver(w.problem, precision="fp32_dc") as s:
        infos, stt = s.solve(u, w.nsteps)
        assert s.stats()["small_solve"] == 2
    assert stt == 0
    U = host(u)
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
