"""GPU parity of the stabilised preconditioner (RD_PC_STABILIZED: the square of F's Jacobian with
its nonlinear factor replaced by a constant s, Section 3.3's construction of G, for any scalar
reaction) through the C ABI, against the CPU oracles: G^{-1} to 1e-12; FP64 steps with the
oracle's iteration counts and max relative error <= 1e-10; FP32 + FP64 defect correction
<= 1e-9 relative L2; on 2-D band sweeps, the one-launch small solve, 3-D grids and long 2-D
grids; near the equilibria, where G = A_lin^2 diverges, the stabilised steps converge."""
import numpy as np
import pytest

from oracle import rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL
from parity_util import assert_same_iterations

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


CASES = [("allen_cahn", "laplacian", 2.0), ("ch_implicit", "neg_biharmonic", 2.0), ("ch_split", "neg_biharmonic", 3.0)]
# (nz, ny, nx): band sweeps, small-solve sized, 3-D, a long 2-D side
SHAPES = [(1, 32, 64), (1, 64, 64), (1, 128, 256), (8, 16, 32), (1, 4, 8192)]


def _pb(kind, op, bc, nz, ny, nx, s, **kw):
    lap = op == "laplacian"
    base = dict(nx=nx, ny=ny, nz=nz, lx=1.7 * nx / 64, ly=1.3 * ny / 64, lz=0.8, bc=bc, op=op, kind=kind,
                dt=2e-3 if lap else 1e-5, a=0.05 if lap else 4e-4, b=20.0 if lap else 1.0, tau_u=0.9,
                tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=5000, precond="stabilized", shift=s)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
@pytest.mark.parametrize("shape", SHAPES)
def test_stabilized_preconditioner_solve_matches_oracle(bc, kind, op, s, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape, s)
    W = WL.rng(21).standard_normal(pb.shape)
    with rd.Solver(pb) as sv:
        y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        sv.apply_precond(dev(W), y)
        got = host(y)
    assert rel_max(got, O.apply_ginv(pb, W)) <= 1e-12


def _gpu_measure_at(pb, uk):
    rd = _rd()

    def at(m):
        with rd.Solver(pb.replace(max_iter=m)) as sv:
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = sv.step(dev(uk), out, allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED))
        return info["residual"]
    return at


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,s", CASES)
@pytest.mark.parametrize("shape", SHAPES)
def test_stabilized_steps_match_oracle(bc, kind, op, s, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape, s)
    uk = WL.rng(22).uniform(-0.9, 0.9, pb.shape)
    U_ref, info_ref = O.pdhg_step(pb, uk, history=True)
    assert info_ref["status"] == O.OK
    with rd.Solver(pb) as sv:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = sv.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0, info
    assert_same_iterations(info["iterations"], info_ref, pb, uk, _gpu_measure_at(pb, uk))
    assert rel_max(U, U_ref) <= 1e-10
    with rd.Solver(pb, precision="fp32_dc") as sv:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = sv.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0, info
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


@pytest.mark.parametrize("kind,op,kw", [
    ("allen_cahn", "laplacian", dict(a=0.1, b=10.0, dt=0.05)),
    ("ch_implicit", "neg_biharmonic", dict(a=4e-4, b=1.0, dt=1e-4, lx=1.0, ly=1.0)),
])
@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_stabilized_converges_where_the_linear_G_diverges(kind, op, kw, precision):
    rd = _rd()
    n = 64
    x = np.arange(n) * 2 * np.pi / n
    u0 = np.tanh(3 * np.sin(x)[None, :] * np.cos(x)[:, None])[None]
    base = dict(nx=n, ny=n, lx=2 * np.pi, ly=2 * np.pi, bc="periodic", op=op, kind=kind, tau_u=1.0, tau_p=1.0,
                tol=1e-10, tol_kind="f_rel", shift=2.0, max_iter=3000)
    base.update(kw)
    lin, stab = WL.Problem(precond="linear", **base), WL.Problem(precond="stabilized", **base)
    _, info_lin = O.pdhg_step(lin, u0)
    U_ref, info_ref = O.pdhg_step(stab, u0)
    assert info_lin["status"] == O.DIVERGED and info_ref["status"] == O.OK
    with rd.Solver(lin, precision=precision) as sv:
        out = torch.empty(lin.shape, dtype=torch.float64, device="cuda")
        info = sv.step(dev(u0), out, allow=(rd.RD_ERR_DIVERGED, rd.RD_ERR_NOT_CONVERGED))
    assert info["status"] != 0
    with rd.Solver(stab, precision=precision) as sv:
        out = torch.empty(stab.shape, dtype=torch.float64, device="cuda")
        info = sv.step(dev(u0), out)
        U = host(out)
    assert info["status"] == 0, info
    if precision == "fp64":
        assert rel_max(U, U_ref) <= 1e-10
    else:
        assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_stabilized_refused_for_two_species():
    rd = _rd()
    gs = WL.Problem(nx=16, ny=16, lx=1.0, ly=1.0, bc="periodic", op="laplacian", kind="gray_scott",
                    p=(2e-3, 1e-3, 0.04, 0.06), dt=1.0, precond="stabilized", shift=2.0)
    with pytest.raises(rd.RDError) as e:
        rd.Solver(gs)
    assert e.value.status == rd.RD_ERR_UNSUPPORTED
