"""GPU parity on 2-D grids with a side longer than the band / column sweeps transform (above 2048
points in FP32, 4096 in FP64, up to 8192): these run on the line-transform kernels with nz = 1
(pointwise residual and update, the x transform, the y transform with the spectral scaling, the
inverse x transform with the dual update), lines of 4096 and 8192 points on blocks of n / 8
threads.  Element by element against the CPU oracles on the same seeded inputs, through the
C ABI; tolerances as for every 2-D grid:
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
    ("allen_cahn", "laplacian"),
    ("ch_implicit", "neg_biharmonic"),
    ("ch_split", "neg_biharmonic"),
]
# (ny, nx): a long x side, a long y side, both long sides of the two lengths
FP64_SHAPES = [(4, 8192), (8192, 2), (16, 8192), (8192, 32)]
FP32_SHAPES = [(8, 4096), (4096, 16), (4, 8192), (8192, 8), (64, 8192)]


def _pb(kind, op, bc, ny, nx, scaled=False, **kw):
    """scaled: side lengths in proportion to the points (h about 0.02 as on a 64^2 grid of the
    same lengths), so that the nonlinear terms stay as stiff as on the small grids and a step
    converges to the tolerance; otherwise [0,1.7) x [0,1.3) whatever the points."""
    ch = op == "neg_biharmonic"
    lx, ly = (1.7 * nx / 64, 1.3 * ny / 64) if scaled else (1.7, 1.3)
    base = dict(nx=nx, ny=ny, lx=lx, ly=ly, bc=bc, op=op, kind=kind,
                dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                tau_u=0.9, tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=3000)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op", KINDS)
@pytest.mark.parametrize("shape", FP64_SHAPES)
def test_long_residual_matches_oracle(bc, kind, op, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    r = WL.rng(11)
    U, Uk = r.uniform(-0.8, 0.8, pb.shape), r.uniform(-0.8, 0.8, pb.shape)
    with rd.Solver(pb) as s:
        assert s.stats()["line_kernels"] == 1
        w = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.residual(dev(U), dev(Uk), w)
        got = host(w)
    assert rel_max(got, O.residual(pb, U, Uk)) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op", KINDS)
@pytest.mark.parametrize("shape", FP64_SHAPES)
def test_long_preconditioner_solve_matches_oracle(bc, kind, op, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape)
    W = WL.rng(12).standard_normal(pb.shape)
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
    ("allen_cahn", "laplacian", "periodic", (8, 8192)),
    ("allen_cahn", "laplacian", "neumann", (8192, 4)),
    ("ch_split", "neg_biharmonic", "periodic", (8192, 8)),
    ("ch_implicit", "neg_biharmonic", "neumann", (4, 8192)),
]


@pytest.mark.parametrize("kind,op,bc,shape", STEP_CASES)
@pytest.mark.parametrize("loop", ["graph", "host"])
def test_long_fp64_step_matches_oracle(kind, op, bc, shape, loop):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape, scaled=True)
    uk = WL.rng(13).uniform(-0.8, 0.8, pb.shape)
    U_ref, info_ref = O.pdhg_step(pb, uk, history=True)
    with rd.Solver(pb, solve_loop=loop) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0 and info_ref["status"] == O.OK
    assert_same_iterations(info["iterations"], info_ref, pb, uk, _gpu_measure_at(pb, uk))
    assert rel_max(U, U_ref) <= 1e-10
    assert abs(info["mass"] - O.mass(pb, U_ref)) <= 1e-12 * max(1.0, abs(O.mass(pb, U_ref)))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op", [("allen_cahn", "laplacian"), ("ch_split", "neg_biharmonic")])
@pytest.mark.parametrize("shape", FP32_SHAPES)
def test_long_fp32_defect_correction_step_matches_oracle(bc, kind, op, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, *shape, scaled=True)
    uk = WL.rng(14).uniform(-0.8, 0.8, pb.shape)
    U_ref, _ = O.pdhg_step(pb, uk)
    with rd.Solver(pb, precision="fp32_dc") as s:
        assert s.stats()["line_kernels"] == 1
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0, info
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_long_sides_below_the_limit_stay_on_the_band_sweeps():
    rd = _rd()
    for prec, shape in (("fp32_dc", (16, 2048)), ("fp64", (8, 4096))):
        with rd.Solver(_pb("allen_cahn", "laplacian", "periodic", *shape), precision=prec) as s:
            assert s.stats()["line_kernels"] == 0


def test_long_two_species_and_oversized_refused():
    rd = _rd()
    gs = _pb("gray_scott", "laplacian", "periodic", 8, 8192, p=(2e-3, 1e-3, 0.04, 0.06), dt=1.0)
    with pytest.raises(rd.RDError) as e:
        rd.Solver(gs, precision="fp32_dc")
    assert e.value.status == rd.RD_ERR_UNSUPPORTED
    with pytest.raises(rd.RDError) as e:
        rd.Solver(_pb("allen_cahn", "laplacian", "periodic", 2, 16384))
    assert e.value.status == rd.RD_ERR_UNSUPPORTED


def test_roofline_sweep_grid_8192_squared_step_matches_oracle():
    """The roofline sweep's grid, Allen-Cahn periodic 8192^2 (the 64^2 configuration's physics), one
    implicit step from its seeded state in both precisions, element by element against the C++
    oracle on all host cores.  The step diffuses the i.i.d. initial state to 1/140 of its norm, so
    the threshold, relative to ||U^k||, is tightened to 1e-13: at 1e-11 two solutions within it
    (the oracle's and defect correction's, which take different paths to it) may differ by
    about 1.4e-9 of ||U^{k+1}|| (measured: 1.0e-9), above the per-step bound the test checks."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic_8192()
    pb = w.problem.replace(tol=1e-13, tol_kind="f_rel", max_iter=10000)
    C.set_threads(0)
    U_ref, info_ref = C.pdhg_step(pb, w.u0)
    assert info_ref["status"] == C.OK
    for prec in ("fp64", "fp32_dc"):
        u = dev(w.u0)
        with rd.Solver(pb, precision=prec) as s:
            assert s.stats()["line_kernels"] == 1
            info = s.step(u, u)
        assert info["status"] == 0, info
        U = host(u)
        del u
        if prec == "fp64":
            assert abs(info["iterations"] - info_ref["iterations"]) <= 1
            assert rel_max(U, U_ref) <= 1e-10
        else:
            assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
        print({"precision": prec, "iterations": info["iterations"], "oracle_iterations": info_ref["iterations"],
               "max_rel": rel_max(U, U_ref), "rel_l2": float(np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref))})


def test_roofline_sweep_fixed_iterations():
    """The sweep's fixed-iteration form (threshold 0, max_iter = 200): both precisions run exactly
    200 PDHG updates and report not converged; FP64 leaves U_200, which equals the oracle's."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic_8192(n=512, fixed_iters=20)
    pb = w.problem
    U_ref, info_ref = O.pdhg_step(pb, w.u0)
    assert info_ref["status"] == O.NOT_CONVERGED and info_ref["iterations"] == 20
    u = dev(w.u0)
    out = torch.empty_like(u)
    with rd.Solver(pb) as s:
        info = s.step(u, out, allow=(rd.RD_ERR_NOT_CONVERGED,))
    assert info["iterations"] == 20
    assert rel_max(host(out), U_ref) <= 1e-10
    with rd.Solver(pb, precision="fp32_dc", dc_max_outer=1, dc_stall_window=1 << 30, dc_inner_rtol=1e-300) as s:
        info = s.step(u, out, allow=(rd.RD_ERR_NOT_CONVERGED,))
    assert info["iterations"] == 20
