"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle, element by element,
on the same seeded inputs.

Tolerances (from the arithmetic of each path):
  * single operators (F, G^{-1}) in FP64: 1e-12 relative to the largest magnitude;
  * a converged FP64 step: the same iteration count as the oracle (off by one only at a rounding
    tie of the stopping measure, tests/parity_util.py) and max |U_gpu - U_ref| <= 1e-10 max |U_ref|;
  * the FP32 + FP64 defect-correction path: relative L2 error <= 1e-9 per step.
"""
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


KINDS = [
    ("none", "laplacian", ()),
    ("none", "neg_biharmonic", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("ch_split", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
]
SHAPES = [(2, 2), (4, 8), (16, 16), (32, 64), (128, 64), (256, 256)]


def _problem(kind, op, p, bc, ny, nx, **kw):
    ch = op == "neg_biharmonic"
    base = dict(nx=nx, ny=ny, lx=1.0, ly=1.3, bc=bc, op=op, kind=kind, p=p,
                dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                tau_u=0.9, tau_p=0.9, tol=1e-12, tol_kind="f_rel", max_iter=3000)
    base.update(kw)
    return WL.Problem(**base)


def _state(pb, seed):
    r = WL.rng(seed)
    if pb.kind == "gray_scott":
        return np.stack([1 - 0.5 * r.random((pb.ny, pb.nx)), 0.25 * r.random((pb.ny, pb.nx))])
    if pb.kind == "schnakenberg":
        return WL.schnakenberg_initial(pb.nx)[:, :pb.ny, :] * (1 + 0.05 * r.uniform(-1, 1, pb.shape)) \
            if pb.nx == pb.ny else 0.9 + 0.1 * r.random(pb.shape)
    return r.uniform(-0.8, 0.8, pb.shape)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", KINDS)
@pytest.mark.parametrize("shape", SHAPES)
def test_residual_map_matches_oracle(bc, kind, op, p, shape):
    """W = F(U) (eq. F(U) rd equation, F(U) CH, Section 3.4.1) on the GPU in FP64."""
    rd = _rd()
    pb = _problem(kind, op, p, bc, *shape)
    U, Uk = _state(pb, 1), _state(pb, 2)
    with rd.Solver(pb) as s:
        w = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.residual(dev(U), dev(Uk), w)
        got = host(w)
    want = O.residual(pb, U, Uk)
    assert rel_max(got, want) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", KINDS)
@pytest.mark.parametrize("shape", SHAPES)
def test_preconditioner_solve_matches_oracle(bc, kind, op, p, shape):
    """Y = G^{-1} W through the GPU Hartley / DCT-II transforms vs the oracle's FFT / DCT."""
    rd = _rd()
    pb = _problem(kind, op, p, bc, *shape)
    W = WL.rng(5).standard_normal(pb.shape)
    with rd.Solver(pb) as s:
        y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.apply_precond(dev(W), y)
        got = host(y)
    want = O.apply_ginv(pb, W)
    assert rel_max(got, want) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("band_rows,col_width", [(0, 0), (6, 8), (2, 2), (10, 32)])
def test_ragged_tiles_preconditioner(bc, band_rows, col_width):
    """Row bands that do not divide ny (ragged last band) and several column-block widths."""
    rd = _rd()
    pb = _problem("allen_cahn", "laplacian", (), bc, 64, 128)
    W = WL.rng(6).standard_normal(pb.shape)
    with rd.Solver(pb, band_rows=band_rows, col_width=col_width) as s:
        y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        s.apply_precond(dev(W), y)
        got = host(y)
    assert rel_max(got, O.apply_ginv(pb, W)) <= 1e-12


def _gpu_measure_at(pb, uk, precision="fp64", **opts):
    """The GPU's stopping measure of its iterate m: a step capped at m updates."""
    rd = _rd()

    def at(m):
        with rd.Solver(pb.replace(max_iter=m), precision=precision, **opts) as s:
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = s.step(dev(uk), out, allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED))
        assert info["iterations"] == m, info
        return info["residual"]
    return at


def _compare_step(pb, uk, precision="fp64", **opts):
    rd = _rd()
    U_ref, info_ref = O.pdhg_step(pb, uk, history=True)
    with rd.Solver(pb, precision=precision, **opts) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out, allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED, rd.RD_ERR_DIVERGED))
        U = host(out)
    return U, info, U_ref, info_ref


STEP_CASES = [
    ("allen_cahn", "laplacian", (), "periodic", (64, 64)),
    ("allen_cahn", "laplacian", (), "neumann", (32, 128)),
    ("ch_implicit", "neg_biharmonic", (), "periodic", (64, 64)),
    ("ch_split", "neg_biharmonic", (), "neumann", (64, 32)),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic", (64, 64)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695), "neumann", (64, 64)),
    ("none", "laplacian", (), "neumann", (16, 16)),
]


@pytest.mark.parametrize("kind,op,p,bc,shape", STEP_CASES)
def test_fp64_step_matches_oracle(kind, op, p, bc, shape):
    """One implicit step in FP64: same PDHG iteration count and <= 1e-10 max relative error."""
    pb = _problem(kind, op, p, bc, *shape)
    uk = _state(pb, 3)
    U, info, U_ref, info_ref = _compare_step(pb, uk)
    assert info["status"] == 0 and info_ref["status"] == O.OK
    assert_same_iterations(info["iterations"], info_ref, pb, uk, _gpu_measure_at(pb, uk))
    assert rel_max(U, U_ref) <= 1e-10


@pytest.mark.parametrize("kind,op,p,bc,shape", STEP_CASES)
def test_fp32_defect_correction_step_matches_oracle(kind, op, p, bc, shape):
    """FP32 PDHG sweeps + FP64 defect correction: relative L2 error <= 1e-9 against the oracle."""
    pb = _problem(kind, op, p, bc, *shape)
    uk = _state(pb, 4)
    U, info, U_ref, _ = _compare_step(pb, uk, precision="fp32_dc")
    assert info["status"] == 0, info
    assert info["outer_rounds"] >= 2
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_allen_cahn_64_periodic_twenty_steps():
    """Allen-Cahn periodic 64x64 on [0,2pi)^2, eps=0.1, dt=0.01, 20 steps, ||Res||_2 <= 1e-10:
    per-step iteration counts equal the oracle's and the final state agrees to 1e-10."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic()
    U_ref, infos_ref = O.solve(w.problem, w.u0, w.nsteps)
    u = dev(w.u0)
    with rd.Solver(w.problem) as s:
        infos, st = s.solve(u, w.nsteps)
    U = host(u)
    assert st == 0
    assert [i["iterations"] for i in infos] == [i["iterations"] for i in infos_ref]
    assert rel_max(U, U_ref) <= 1e-10


def test_not_converged_and_diverged_statuses():
    rd = _rd()
    pb = _problem("allen_cahn", "laplacian", (), "periodic", 32, 32, max_iter=3)
    uk = _state(pb, 7)
    U, info, U_ref, info_ref = _compare_step(pb, uk)
    assert info["status"] == rd.RD_ERR_NOT_CONVERGED and info["iterations"] == 3
    assert info_ref["status"] == O.NOT_CONVERGED
    assert rel_max(U, U_ref) <= 1e-12
    pb = _problem("none", "laplacian", (), "periodic", 32, 32, tau_u=1.4, tau_p=1.0, max_iter=100000)
    U, info, U_ref, info_ref = _compare_step(pb, uk)
    assert info["status"] == rd.RD_ERR_DIVERGED and info_ref["status"] == O.DIVERGED
    assert info["iterations"] == info_ref["iterations"]


def test_solve_host_buffers_match_device_solve():
    rd = _rd()
    w = WL.config_allen_cahn_neumann(64, 3, seed=11)
    u = dev(w.u0)
    uh = np.ascontiguousarray(w.u0.copy())
    with rd.Solver(w.problem) as s:
        s.solve(u, 3)
        s.solve_host(uh, 3)
    assert np.array_equal(host(u), uh)


def test_step_in_place_alias():
    rd = _rd()
    pb = _problem("ch_split", "neg_biharmonic", (), "periodic", 32, 32)
    uk = _state(pb, 8)
    U_ref, _ = O.pdhg_step(pb, uk)
    u = dev(uk)
    with rd.Solver(pb) as s:
        s.step(u, u)
    assert rel_max(host(u), U_ref) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
@pytest.mark.parametrize("kind,op,p,bc,shape", [STEP_CASES[1], STEP_CASES[3], STEP_CASES[4]])
def test_transform_buffer_modes_agree(precision, kind, op, p, bc, shape):
    """In-place (one buffer) and ping-pong (two buffers) shared-memory transforms perform the same
    arithmetic: the steps agree bit for bit, and both match the oracle."""
    pb = _problem(kind, op, p, bc, *shape)
    uk = _state(pb, 9)
    outs = []
    for fb in (1, 2):
        U, info, U_ref, _ = _compare_step(pb, uk, precision=precision, fft_buffers=fb)
        assert info["status"] == 0, info
        tol = 1e-10 if precision == "fp64" else 1e-9
        assert np.linalg.norm(U - U_ref) <= tol * np.linalg.norm(U_ref)
        outs.append(U)
    assert np.array_equal(outs[0], outs[1])


BENCH_WORKLOADS = {
    "allen_cahn_neumann_1024": lambda: WL.config_allen_cahn_neumann(),
    "cahn_hilliard_split_512": lambda: WL.config_cahn_hilliard_split(),
    "gray_scott_2048": lambda: WL.config_gray_scott(),
    "schnakenberg_128": lambda: WL.config_schnakenberg(),
    "allen_cahn_periodic_64": lambda: WL.config_allen_cahn_periodic(),
}


def _apply_g(pb, Y):
    """G Y with G = A_lin^2 applied as stencils (oracle five-point Laplacian), per component."""
    out = np.empty_like(Y)
    for c in range(pb.ncomp):
        if pb.kind in ("gray_scott", "schnakenberg"):
            A = lambda v, D=pb.p[c]: v - D * pb.dt * O.lap(v, pb)
        elif pb.op == "laplacian":
            A = lambda v: v - pb.a * pb.dt * O.lap(v, pb)
        else:
            A = lambda v: v + pb.a * pb.dt * O.lap(O.lap(v, pb), pb)
        out[c] = A(A(Y[c]))
    return out


@pytest.mark.parametrize("name", sorted(BENCH_WORKLOADS))
@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_benchmark_workloads_plan_in_both_precisions(name, precision):
    """Every benchmarked workload finds a launch plan that fits shared memory in both precisions.
    FP64: the preconditioner solve at that size against the oracle up to 512^2 points, above that
    through G Y = W with G applied back as stencils.  FP32 defect correction: one step from the
    workload's initial state meets the stopping rule, with F evaluated by the oracle."""
    rd = _rd()
    w = BENCH_WORKLOADS[name]()
    pb = w.problem
    if precision == "fp64":
        W = WL.rng(12).standard_normal(pb.shape)
        with rd.Solver(pb, precision=precision) as s:
            y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            s.apply_precond(dev(W), y)
            got = host(y)
        if pb.nx * pb.ny <= 512 * 512:
            assert rel_max(got, O.apply_ginv(pb, W)) <= 1e-12
        else:
            assert rel_max(_apply_g(pb, got), W) <= 1e-10
    else:
        with rd.Solver(pb, precision=precision) as s:
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = s.step(dev(w.u0), out)
            U = host(out)
        assert info["status"] == 0, info
        r, thr = O.measure(pb, O.residual(pb, U, w.u0), w.u0)
        assert r <= thr * (1 + 1e-6), (r, thr)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_device_loop_trip_length_does_not_change_results(precision):
    """The device-side loop runs graph_k iterations per trip and stops itself: the trip length
    changes neither the iterates (bit for bit) nor the iteration counts."""
    rd = _rd()
    pb = _problem("allen_cahn", "laplacian", (), "neumann", 64, 64)
    uk = _state(pb, 10)
    outs, infos = [], []
    for gk in (1, 3, 8):
        U, info, U_ref, info_ref = _compare_step(pb, uk, precision=precision, graph_k=gk)
        assert info["status"] == 0, info
        outs.append(U)
        infos.append((info["iterations"], info["outer_rounds"]))
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    assert len(set(infos)) == 1


def test_host_syncs_per_step():
    """One graph launch and one host read per step: FP64 (the PDHG loop on the device) and
    defect correction, whose outer rounds loop on the device too (a WHILE node over the rounds,
    each holding the inner solve: one launch, or a nested WHILE node)."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic(64, 3)
    for precision, small in (("fp64", 0), ("fp32_dc", 0), ("fp32_dc", 1)):
        u = dev(w.u0)
        with rd.Solver(w.problem, precision=precision, small_solve=small) as s:
            assert s.stats()["small_solve"] == (2 if small else 0)
            s.reset_stats()
            infos, st = s.solve(u, 3)
            stats = s.stats()
        assert st == 0
        assert stats["host_syncs"] == 3 and stats["graph_launches"] == 3
        if precision == "fp32_dc":
            assert stats["residual_passes"] == sum(i["outer_rounds"] for i in infos)
        assert stats["pdhg_iterations"] == sum(i["iterations"] for i in infos)


def test_defect_correction_outer_round_limit():
    """dc_max_outer = 1: one inner solve, two FP64 residual evaluations, then NOT_CONVERGED
    with the iterate after that one correction (the FP64 plain step converges to it only later)."""
    rd = _rd()
    pb = _problem("allen_cahn", "laplacian", (), "periodic", 32, 32)
    uk = _state(pb, 11)
    with rd.Solver(pb, precision="fp32_dc", dc_max_outer=1) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out, allow=(rd.RD_OK, rd.RD_ERR_NOT_CONVERGED))
    assert info["status"] == rd.RD_ERR_NOT_CONVERGED
    assert info["outer_rounds"] == 2 and info["iterations"] > 0


@pytest.mark.parametrize("precision,fused", [("fp64", 0), ("fp32_dc", 0), ("fp32_dc", 1)])
@pytest.mark.parametrize("kind,op,p,bc,shape", [STEP_CASES[1], STEP_CASES[3], STEP_CASES[4]])
def test_host_loop_matches_graph_loop(precision, fused, kind, op, p, bc, shape):
    """The host-relaunched loop (plain graphs, for profilers) runs the same kernels in the same
    order as the device-side WHILE loop, unfused or with the fused update: bit-identical steps
    and the same iteration and round counts."""
    rd = _rd()
    pb = _problem(kind, op, p, bc, *shape)
    uk = _state(pb, 13)
    res = []
    for loop in ("graph", "host"):
        # small_solve = 0: these grids would otherwise run each inner solve in one launch
        with rd.Solver(pb, precision=precision, solve_loop=loop, fused_update=fused, small_solve=0) as s:
            assert s.stats()["fused_update"] == fused
            out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            info = s.step(dev(uk), out)
            U = host(out)
        assert info["status"] == 0, info
        res.append((U, info["iterations"], info["outer_rounds"]))
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1:] == res[1][1:]


@pytest.mark.parametrize("fft_unrolled", [0, 1])
@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_transform_pass_forms_match_oracle(fft_unrolled, bc):
    """Looped and length-specialised unrolled transform passes: the preconditioner solve in FP64
    within 1e-12 of the oracle on every line length 64 .. 2048, and one defect-corrected step."""
    rd = _rd()
    shapes = [(n, n) for n in (64, 128, 256)] + [(8, n) for n in (512, 1024, 2048)] + [(n, 8) for n in (512, 2048)]
    for ny, n in shapes:
        pb = _problem("allen_cahn", "laplacian", (), bc, ny, n)
        W = WL.rng(14).standard_normal(pb.shape)
        with rd.Solver(pb, fft_unrolled=fft_unrolled) as s:
            y = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
            s.apply_precond(dev(W), y)
            got = host(y)
        assert rel_max(got, O.apply_ginv(pb, W)) <= 1e-12, n
    pb = _problem("ch_split", "neg_biharmonic", (), bc, 64, 64)
    uk = _state(pb, 15)
    U, info, U_ref, _ = _compare_step(pb, uk, precision="fp32_dc", fft_unrolled=fft_unrolled)
    assert info["status"] == 0, info
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
def test_autotuned_tiles_match_oracle(precision):
    """The autotuner times the candidate tile shapes at create and keeps one that fits (the
    residual and update sweeps may get different band heights); the step it then takes matches
    the oracle within the usual tolerances."""
    rd = _rd()
    pb = _problem("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic", 64, 128)
    uk = _state(pb, 16)
    U_ref, info_ref = O.pdhg_step(pb, uk)
    with rd.Solver(pb, precision=precision, autotune=1) as s:
        st = s.stats()
        assert st["plan_band_rows"] in (2, 4, 8, 16) and st["plan_upd_rows"] in (2, 4, 8, 16)
        assert st["plan_col_width"] in (2, 4, 8, 16, 32, 64)
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    assert info["status"] == 0, info
    tol = 1e-10 if precision == "fp64" else 1e-9
    assert np.linalg.norm(U - U_ref) <= tol * np.linalg.norm(U_ref)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("res_rows,upd_rows", [(2, 8), (8, 2), (4, 16)])
def test_different_band_heights_for_residual_and_update(bc, res_rows, upd_rows):
    """k_res and k_upd with different band heights (as the autotuner may choose) give a step that
    matches the oracle and agrees with one common height to rounding of the norm partials."""
    rd = _rd()
    pb = _problem("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), bc, 64, 64)
    uk = _state(pb, 17)
    U_ref, _ = O.pdhg_step(pb, uk)
    res = []
    for u_rows in (upd_rows, res_rows):
        U, info, _, _ = _compare_step(pb, uk, precision="fp32_dc", band_rows=res_rows, upd_rows=u_rows)
        assert info["status"] == 0, info
        assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
        res.append(U)
    assert np.linalg.norm(res[0] - res[1]) <= 1e-10 * np.linalg.norm(U_ref)


FUSED_CASES = [
    ("allen_cahn", "laplacian", (), "periodic", (64, 64)),
    ("allen_cahn", "laplacian", (), "neumann", (32, 128)),
    ("ch_split", "neg_biharmonic", (), "neumann", (64, 32)),
    ("ch_implicit", "neg_biharmonic", (), "periodic", (64, 64)),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic", (64, 64)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695), "neumann", (64, 64)),
]


@pytest.mark.parametrize("kind,op,p,bc,shape", FUSED_CASES)
@pytest.mark.parametrize("upd_rows", [2, 4])
def test_fused_update_matches_oracle(kind, op, p, bc, shape, upd_rows):
    """The fused update + residual kernel (per-band halo copies of U, ping-pong transform buffer)
    gives a defect-corrected step within 1e-9 of the oracle, with several bands per grid."""
    pb = _problem(kind, op, p, bc, *shape)
    uk = _state(pb, 18)
    rd = _rd()
    with rd.Solver(pb, precision="fp32_dc", fused_update=1, upd_rows=upd_rows, small_solve=0) as s:
        assert s.stats()["fused_update"] == 1
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out)
        U = host(out)
    U_ref, _ = O.pdhg_step(pb, uk)
    assert info["status"] == 0, info
    assert info["outer_rounds"] >= 2
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_fused_update_twenty_steps_match_unfused():
    """Allen-Cahn periodic 64^2, 20 steps: the fused and unfused loops agree to the step
    tolerance (their FP32 inner iterates differ only by rounding)."""
    rd = _rd()
    w = WL.config_allen_cahn_periodic()
    outs = []
    for fu in (0, 1):
        w = WL.config_allen_cahn_periodic()
        pb = w.problem.replace(tol_kind="f_rel", tol=1e-11)
        u = dev(w.u0)
        with rd.Solver(pb, precision="fp32_dc", fused_update=fu, small_solve=0) as s:
            assert s.stats()["fused_update"] == fu
            infos, st = s.solve(u, w.nsteps)
        assert st == 0
        outs.append(host(u))
    assert rel_max(outs[1], outs[0]) <= 1e-9


@pytest.mark.parametrize("name", ["allen_cahn_neumann_1024", "cahn_hilliard_split_512", "gray_scott_2048"])
def test_benchmark_workloads_in_the_bench_launch_configuration(name):
    """The benchmarked workloads at full size in the configuration bench.py times (tiles and the
    fused update chosen by the autotuner, the device-side loop): three steps from the initial
    state, each meeting the stopping rule with F evaluated by the oracle from the GPU's U^k and
    U^{k+1}, and the iteration counts reported per step."""
    rd = _rd()
    w = BENCH_WORKLOADS[name]()
    pb = w.problem
    u = dev(w.u0)
    with rd.Solver(pb, precision="fp32_dc", autotune=1, fused_update=1) as s:
        for _ in range(3):
            uk = host(u)
            info = s.step(u, u)
            U = host(u)
            assert info["status"] == 0 and info["iterations"] > 0, info
            r, thr = O.measure(pb, O.residual(pb, U, uk), uk)
            assert r <= thr * (1 + 1e-6), (r, thr)


def test_defect_correction_stall_window_escalates():
    """A request of the serving mix (Allen-Cahn Neumann 64^2, 49 steps, ||F|| <= 1e-6 ||U^k||)
    whose step 47 converges slowly: with a fixed stall window the FP32 inner solves were cut off
    before they made progress and the step ran out of outer rounds.  The window now doubles after
    an outer round that does not halve the FP64 residual, so every step converges, alone and in a
    batch, and the result agrees with the plain FP64 solve to the tolerance."""
    rd = _rd()
    pb, u0, n = WL.serving_requests(456, 5000)[455]
    assert (pb.kind, pb.bc, pb.nx, n) == ("allen_cahn", "neumann", 64, 49)
    outs = {}
    for prec in ("fp32_dc", "fp64"):
        u = dev(u0)
        with rd.Solver(pb, precision=prec) as s:
            infos, st = s.solve(u, n)
        assert st == 0 and all(i["status"] == 0 for i in infos)
        outs[prec] = host(u)
    assert np.linalg.norm(outs["fp32_dc"] - outs["fp64"]) <= 1e-5 * np.linalg.norm(outs["fp64"])
    with rd.Batch(1 << 28, 4) as b:
        rid, out = b.submit(pb, u0, n)
        res = []
        while not res:
            res = b.poll(timeout=5.0)
    assert res[0]["status"] == 0 and res[0]["steps"] == n, res[0]
    assert np.linalg.norm(out - outs["fp64"]) <= 1e-5 * np.linalg.norm(outs["fp64"])
