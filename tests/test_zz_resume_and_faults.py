"""Checkpoint and resume, and a non-finite input, on the GPU through the C ABI.

Between implicit steps a solve's whole state is U^k: each step restarts from U_0 = U^k, P_0 = 0
(Section 2.1, "Initial guess"; Algorithm 1), and everything else is fixed at create.  So a run of
2 + 2 steps with the state written to a file and read back into a NEW handle in between is, bit
for bit, the run of 4 steps on one handle, with the same iteration counts per step: FP64 and
defect correction, on the one-launch small solve, the band sweeps and a 3-D grid.

A NaN in U^k makes the first stopping measure non-finite: the step ends as diverged before any
update, as in the oracle, on every path and in a batch next to a request that converges."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
@pytest.mark.parametrize("kind,op,bc,shape", [
    ("allen_cahn", "laplacian", "periodic", (1, 32, 64)),
    ("ch_split", "neg_biharmonic", "neumann", (1, 128, 256)),
    ("allen_cahn", "laplacian", "neumann", (8, 16, 16)),
])
def test_resume_from_a_checkpoint_equals_the_uninterrupted_run(tmp_path, precision, kind, op, bc, shape):
    rd = _rd()
    nz, ny, nx = shape
    ch = op == "neg_biharmonic"
    pb = WL.Problem(nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.3, lz=0.7, bc=bc, op=op, kind=kind,
                    dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                    tau_u=0.9, tau_p=0.9, tol=1e-11, tol_kind="f_rel", max_iter=3000)
    u0 = WL.rng(60).uniform(-0.8, 0.8, pb.shape)
    u = dev(u0)
    with rd.Solver(pb, precision=precision) as s:
        infos, status = s.solve(u, 4)
    assert status == 0
    whole = host(u)
    v = dev(u0)
    with rd.Solver(pb, precision=precision) as s:
        first, status = s.solve(v, 2)
    assert status == 0
    ckpt = tmp_path / "u.npy"
    np.save(ckpt, host(v))
    del v
    w = dev(np.load(ckpt))
    with rd.Solver(pb, precision=precision) as s:
        second, status = s.solve(w, 2)
    assert status == 0
    assert np.array_equal(host(w), whole)
    assert [i["iterations"] for i in first + second] == [i["iterations"] for i in infos]


CASES = [("allen_cahn", "laplacian", "periodic", (1, 32, 64)),
         ("ch_split", "neg_biharmonic", "neumann", (1, 128, 256)),
         ("allen_cahn", "laplacian", "neumann", (8, 16, 16))]


def _pb(kind, op, bc, shape):
    nz, ny, nx = shape
    ch = op == "neg_biharmonic"
    return WL.Problem(nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.3, lz=0.7, bc=bc, op=op, kind=kind,
                      dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                      tau_u=0.9, tau_p=0.9, tol=1e-11, tol_kind="f_rel", max_iter=3000)


@pytest.mark.parametrize("precision", ["fp64", "fp32_dc"])
@pytest.mark.parametrize("kind,op,bc,shape", CASES)
def test_nan_in_the_state_ends_the_step_as_diverged(precision, kind, op, bc, shape):
    rd = _rd()
    pb = _pb(kind, op, bc, shape)
    uk = WL.rng(61).uniform(-0.8, 0.8, pb.shape)
    uk.reshape(-1)[uk.size // 3] = np.nan
    _, info_ref = O.pdhg_step(pb, uk)
    assert info_ref["status"] == O.DIVERGED and info_ref["iterations"] == 0
    with rd.Solver(pb, precision=precision) as s:
        out = torch.empty(pb.shape, dtype=torch.float64, device="cuda")
        info = s.step(dev(uk), out, allow=(rd.RD_ERR_DIVERGED,))
    assert info["status"] == rd.RD_ERR_DIVERGED and info["iterations"] == 0, info


def test_nan_request_fails_alone_in_a_batch():
    rd = _rd()
    good = _pb("allen_cahn", "laplacian", "periodic", (1, 64, 64))
    u_good = WL.rng(62).uniform(-0.8, 0.8, good.shape)
    u_bad = u_good.copy()
    u_bad[0, 5, 7] = np.nan
    results = {}
    with rd.Batch(1 << 30, 4) as b:
        ids = [b.submit(good, u_bad, 2, tag=0)[0], b.submit(good, u_good, 2, tag=1)[0]]
        t0 = time.time()
        while len(results) < 2 and time.time() - t0 < 120:
            for r in b.poll(timeout=1.0):
                results[r["id"]] = r
    assert results[ids[0]]["status"] == rd.RD_ERR_DIVERGED, results[ids[0]]
    assert results[ids[1]]["status"] == 0 and results[ids[1]]["steps"] == 2, results[ids[1]]
