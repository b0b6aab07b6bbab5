"""GPU parity on 3-D grids (the paper's scheme with a third axis: seven-point Laplacian, Lap^2 as
its square, separable transforms along x, y and z) through the C ABI, element by element
against the CPU oracles on the same seeded inputs.  Tolerances as for 2-D grids:
  * F and G^{-1} in FP64: 1e-12 relative to the largest magnitude;
  * a converged FP64 step: the oracle's iteration count (a rounding tie at the threshold aside,
    tests/parity_util.py) and max relative error <= 1e-10;
  * FP32 sweeps + FP64 defect correction: relative L2 error <= 1e-9 per step.
"""
import numpy as np
import pytest

from oracle import cpp_oracle as C, rd_oracle as O
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


KINDS = [
    ("none", "laplacian"),
    ("none", "neg_biharmonic"),
    ("allen_cahn", "laplacian"),
    ("ch_implicit", "neg_biharmonic"),
    ("ch_split", "neg_biharmonic"),
]
SHAPES = [(2, 2, 2), (4, 4, 4), (8, 4, 16), (16, 32, 8), (32, 32, 32)]


def _pb(kind, op, bc, nz, ny, nx, **kw):
    ch = op == "neg_biharmonic"
    base = dict(nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.3, lz=0.8, bc=bc, op=op, kind=kind,
                dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                tau_u=0.9, tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=3000)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op", KINDS)
@pytest.mark.parametrize("shape", SHAPES)
def test_3d_residual_matches_oracle(bc, kind, op, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    r = WL.rng(1)
    U, Uk = r.uniform(-0.8, 0.8, pb.shape), r.uniform(-0.8, 0.8, pb.shape)
    with rd.Solver(pb) as s:
        w = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.residual(dev(U), dev(Uk), w)
        got = host(w)
    assert rel_max(got, O.residual(pb, U, Uk)) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op", [("allen_cahn", "laplacian"), ("ch_split", "neg_biharmonic")])
@pytest.mark.parametrize("shape", SHAPES + [(64, 8, 128), (128, 2, 4)])
def test_3d_preconditioner_solve_matches_oracle(bc, kind, op, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    W = WL.rng(5).standard_normal(pb.shape)
    with rd.Solver(pb) as s:
        y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.apply_precond(dev(W), y)
        got = host(y)
    assert rel_max(got, O.apply_ginv(pb, W)) <= 1e-12


def _gpu_measure_at(pb, uk, precision="fp64"):
    rd = _rd()

    def at(m):
        with rd.Solver(pb.replace(max_iter=m), precision=precision) as s:
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = s.step(dev(uk), out, allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED))
        return info["residual"]
    return at


STEP_CASES = [
    ("allen_cahn", "laplacian", "periodic", (16, 16, 16)),
    ("allen_cahn", "laplacian", "neumann", (8, 32, 16)),
    ("ch_implicit", "neg_biharmonic", "periodic", (16, 8, 16)),
    ("ch_split", "neg_biharmonic", "neumann", (16, 16, 16)),
    ("none", "laplacian", "neumann", (4, 8, 8)),
]


@pytest.mark.parametrize("kind,op,bc,shape", STEP_CASES)
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_3d_fp64_step_matches_oracle(kind, op, bc, shape, loop):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    uk = WL.rng(3).uniform(-0.8, 0.8, pb.shape)
    U_ref, info_ref = O.pdhg_step(pb, uk, history=True)
    with rd.Solver(pb, solve_loop=loop) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0 and info_ref["status"] == O.OK
    assert_same_iterations(info["iterations"], info_ref, pb, uk, _gpu_measure_at(pb, uk))
    assert rel_max(U, U_ref) <= 1e-10
    assert abs(info["mass"] - O.mass(pb, U_ref)) <= 1e-12 * max(1.0, abs(O.mass(pb, U_ref)))


@pytest.mark.parametrize("kind,op,bc,shape", STEP_CASES)
def test_3d_fp32_defect_correction_step_matches_oracle(kind, op, bc, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    uk = WL.rng(4).uniform(-0.8, 0.8, pb.shape)
    U_ref, _ = O.pdhg_step(pb, uk)
    with rd.Solver(pb, precision="fp32_dc") as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0 and info["outer_rounds"] >= 2, info
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


@pytest.mark.parametrize("kind,op,bc", [("allen_cahn", "laplacian", "periodic"),
                                        ("ch_split", "neg_biharmonic", "neumann")])
def test_3d_128_cubed_steps_match_oracle(kind, op, bc):
    """The 3-D grid of the serving mix, 128^3, with the mix's physics (Allen-Cahn of the 64^2
    configuration on [0,2pi)^3; Cahn-Hilliard split of the 512^2 configuration on [0,1]^3), two
    steps to ||F|| <= 1e-11 ||U^k|| in both precisions against the C++ oracle."""
    rd = _rd()
    n = 128
    if kind == "allen_cahn":
        pb = WL.Problem(nx=n, ny=n, nz=n, lx=2 * np.pi, ly=2 * np.pi, lz=2 * np.pi, bc=bc, op=op, kind=kind,
                        a=0.1, b=10.0, dt=0.01, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
        u0 = WL.uniform_field(77, pb.shape, -0.05, 0.05)
    else:
        pb = WL.Problem(nx=n, ny=n, nz=n, lx=1.0, ly=1.0, lz=1.0, bc=bc, op=op, kind=kind, a=4e-4, b=1.0,
                        dt=1e-5, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
        u0 = WL.zero_mean_uniform(78, pb.shape, 0.1)
    C.set_threads(0)
    refs = [u0]
    for _ in range(2):
        refs.append(C.pdhg_step(pb, refs[-1])[0])
    for prec in ("fp64", "fp32_dc"):
        u = dev(u0)
        with rd.Solver(pb, precision=prec) as s:
            for k in range(2):
                info = s.step(u, u)
                assert info["status"] == 0, info
                U = host(u)
                if prec == "fp64":
                    assert rel_max(U, refs[k + 1]) <= 1e-10
                else:
                    assert np.linalg.norm(U - refs[k + 1]) <= 1e-9 * np.linalg.norm(refs[k + 1])


def test_3d_two_species_refused():
    rd = _rd()
    pb = WL.Problem(nx=8, ny=8, nz=8, lx=1.0, ly=1.0, lz=1.0, bc="periodic", op="laplacian", kind="gray_scott",
                    p=(2e-3, 1e-3, 0.04, 0.06), dt=1.0)
    with pytest.raises(rd.RDError) as e:
        rd.Solver(pb)
    assert e.value.status == rd.RD_ERR_UNSUPPORTED
