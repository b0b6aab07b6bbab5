"""Batched, continuously served runs (rd_batch_*) on the GPU: results against the CPU oracle,
the same request alone and inside a mix of uneven grid sizes, admission under a small HBM
budget."""
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


def _requests():
    """Uneven sizes and both boundary conditions: Allen-Cahn and Cahn-Hilliard."""
    out = []
    for k, (kind, op, bc, ny, nx) in enumerate([
        ("allen_cahn", "laplacian", "periodic", 64, 64),
        ("allen_cahn", "laplacian", "neumann", 32, 128),
        ("ch_split", "neg_biharmonic", "periodic", 128, 128),
        ("ch_implicit", "neg_biharmonic", "neumann", 64, 32),
        ("allen_cahn", "laplacian", "periodic", 256, 256),
        ("none", "laplacian", "neumann", 16, 16),
    ]):
        ch = op == "neg_biharmonic"
        pb = WL.Problem(nx=nx, ny=ny, lx=1.0, ly=1.0, bc=bc, op=op, kind=kind,
                        dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                        tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
        u0 = WL.uniform_field(50 + k, pb.shape, -0.5, 0.5)
        out.append((pb, u0, 3 + k % 2))
    return out


def _run(reqs, budget=1 << 30, slots=16):
    from paper_2305_03945_gb300 import rd
    results, outs = {}, {}
    with rd.Batch(budget, slots) as b:
        ids = []
        for k, (pb, u0, n) in enumerate(reqs):
            rid, out = b.submit(pb, u0, n, tag=k)
            ids.append(rid)
            outs[rid] = out
        t0 = time.time()
        while len(results) < len(ids) and time.time() - t0 < 120:
            for r in b.poll(timeout=1.0):
                results[r["id"]] = r
        stats = b.stats()
    return ids, results, outs, stats


def test_batch_matches_oracle_per_request():
    reqs = _requests()
    ids, results, outs, stats = _run(reqs)
    assert len(results) == len(reqs)
    for rid, (pb, u0, n) in zip(ids, reqs):
        r = results[rid]
        assert r["status"] == 0 and r["steps"] == n, r
        U_ref, _ = O.solve(pb, u0, n)
        err = np.linalg.norm(outs[rid] - U_ref) / np.linalg.norm(U_ref)
        assert err <= 1e-9, (pb.kind, pb.bc, pb.nx, pb.ny, err)
    assert stats["completed"] == len(reqs)


def test_same_result_alone_and_in_the_mix():
    reqs = _requests()
    probe = reqs[2]
    _, res_alone, out_alone, _ = _run([probe])
    ids, res_mix, out_mix, _ = _run(reqs)
    a = next(iter(out_alone.values()))
    m = out_mix[ids[2]]
    assert np.array_equal(a, m)
    assert next(iter(res_alone.values()))["iterations"] == res_mix[ids[2]]["iterations"]


def _long_request(k):
    """A 256^2 Allen-Cahn run of 40 (k = 0) or 120 (k = 1) steps: still on the GPU when the probe
    arrives, and the second one still running when the first has finished."""
    pb = WL.Problem(nx=256, ny=256, lx=1.0, ly=1.0, bc="periodic", op="laplacian",
                    kind="allen_cahn", dt=2e-3, a=0.05, b=20.0, tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
    return pb, WL.uniform_field(70 + k, pb.shape, -0.5, 0.5), 40 if k == 0 else 120


@pytest.mark.parametrize("slots", [8, 2])
def test_request_arriving_while_others_run(slots):
    """Continuous batching: the probe is submitted only once the batch's graph is running the
    other requests (slots = 8: admitted beside them at once; slots = 2: queued until a running
    request frees its slot).  Its result and iteration count are bit-identical to the same
    request served alone."""
    from paper_2305_03945_gb300 import rd
    probe = _requests()[2]
    _, res_alone, out_alone, _ = _run([probe])
    alone = next(iter(res_alone.values()))
    results = {}
    with rd.Batch(1 << 30, slots) as b:
        others = [b.submit(*_long_request(k), tag=k)[0] for k in range(2)]
        t0 = time.time()
        while b.stats()["graph_launches"] < 3 and time.time() - t0 < 60:
            time.sleep(0.002)
        st = b.stats()
        assert st["graph_launches"] >= 3 and st["completed"] == 0, st
        pid, pout = b.submit(*probe, tag=99)
        while len(results) < 3 and time.time() - t0 < 120:
            for r in b.poll(timeout=1.0):
                results[r["id"]] = r
    assert len(results) == 3 and all(r["status"] == 0 for r in results.values()), results
    p = results[pid]
    first, second = results[others[0]], results[others[1]]
    assert first["t_done"] < second["t_done"]
    if slots == 8:
        # a free slot at submission: admitted beside both running requests
        assert p["t_admit"] < first["t_done"]
    else:
        # no free slot at submission: admitted once the shorter request freed its slot, while
        # the longer one kept running
        assert p["t_admit"] >= first["t_done"] - 1e-3 and p["t_admit"] > p["t_submit"]
    assert p["t_admit"] < second["t_done"]
    assert np.array_equal(pout, next(iter(out_alone.values())))
    assert p["iterations"] == alone["iterations"] and p["outer_rounds"] == alone["outer_rounds"]


def test_admission_under_a_small_budget():
    """A budget that holds only a couple of 128^2 slots still serves every request."""
    reqs = [r for r in _requests() if r[0].nx <= 128][:4] * 2
    ids, results, outs, stats = _run(reqs, budget=3 * 128 * 128 * 48 + (8 << 20), slots=8)
    assert len(results) == len(reqs) and all(r["status"] == 0 for r in results.values())
    assert stats["admitted"] == len(reqs)
    assert max(r["t_admit"] - r["t_submit"] for r in results.values()) > 0


def test_request_larger_than_budget_is_refused():
    from paper_2305_03945_gb300 import rd
    pb, u0, n = _requests()[4]  # 256^2
    with rd.Batch(2 << 20, 4) as b:
        with pytest.raises(rd.RDError) as e:
            b.submit(pb, u0, n)
        assert e.value.status == rd.RD_ERR_BUSY


def _requests3():
    """3-D requests (the 7-point scheme) of both kinds and boundary conditions, uneven sizes."""
    out = []
    for k, (kind, op, bc, nz, ny, nx) in enumerate([
        ("allen_cahn", "laplacian", "periodic", 16, 16, 16),
        ("ch_split", "neg_biharmonic", "neumann", 8, 16, 32),
        ("allen_cahn", "laplacian", "neumann", 32, 32, 32),
        ("ch_implicit", "neg_biharmonic", "periodic", 16, 8, 16),
    ]):
        ch = op == "neg_biharmonic"
        pb = WL.Problem(nx=nx, ny=ny, nz=nz, lx=1.0, ly=1.0, lz=1.0, bc=bc, op=op, kind=kind,
                        dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                        tau_u=1.0, tau_p=1.0, tol=1e-11, tol_kind="f_rel")
        out.append((pb, WL.uniform_field(90 + k, pb.shape, -0.5, 0.5), 3 + k % 2))
    return out


def test_batch_with_3d_requests_matches_oracle():
    """2-D and 3-D requests in one batch: every result against the oracle (<= 1e-9 rel. L2)."""
    reqs = _requests3() + _requests()[:3]
    ids, results, outs, stats = _run(reqs)
    assert len(results) == len(reqs)
    for rid, (pb, u0, n) in zip(ids, reqs):
        r = results[rid]
        assert r["status"] == 0 and r["steps"] == n, r
        U_ref, _ = O.solve(pb, u0, n)
        err = np.linalg.norm(outs[rid] - U_ref) / np.linalg.norm(U_ref)
        assert err <= 1e-9, (pb.kind, pb.bc, pb.nz, pb.ny, pb.nx, err)


def test_3d_request_same_alone_and_in_the_mix():
    reqs = _requests3() + _requests()
    probe = reqs[1]
    _, res_alone, out_alone, _ = _run([probe])
    ids, res_mix, out_mix, _ = _run(reqs)
    assert np.array_equal(next(iter(out_alone.values())), out_mix[ids[1]])
    assert next(iter(res_alone.values()))["iterations"] == res_mix[ids[1]]["iterations"]


def test_serving_mix_128_cubed_request_matches_plain_fp64():
    """A 128^3 request of the serving mix, batched, against the plain FP64 solve of the same
    request to the mix's tolerance (||F|| <= 1e-6 ||U^k||)."""
    from paper_2305_03945_gb300 import rd
    reqs = WL.serving_requests(48)
    k = next(i for i, (pb, _, _) in enumerate(reqs) if pb.nz == 128)
    pb, u0, n = reqs[k]
    n = min(n, 5)
    u = torch.from_numpy(u0.copy()).cuda()
    with rd.Solver(pb, precision="fp64") as s:
        s.solve(u, n)
    ref = u.cpu().numpy()
    ids, results, outs, _ = _run([(pb, u0, n)])
    assert results[ids[0]]["status"] == 0
    assert np.linalg.norm(outs[ids[0]] - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("small", [1, 0])
def test_small_slots_one_launch_inner_solves(small):
    """Small 2-D slots (one block below 16 points a side, a cluster of eight blocks up to 16 K
    points) run each inner solve in one launch beside the sweeps of the larger slots: every
    result against the oracle, and a small request bit-identical alone and in the mix."""
    reqs = _requests()
    from paper_2305_03945_gb300 import rd
    results = {}
    with rd.Batch(1 << 30, 16, small_solve=small) as b:
        ids = [b.submit(pb, u0, n, tag=k) for k, (pb, u0, n) in enumerate(reqs)]
        t0 = time.time()
        while len(results) < len(ids) and time.time() - t0 < 120:
            for r in b.poll(timeout=1.0):
                results[r["id"]] = r
    for (rid, out), (pb, u0, n) in zip(ids, reqs):
        r = results[rid]
        assert r["status"] == 0 and r["steps"] == n, r
        U_ref, _ = O.solve(pb, u0, n)
        assert np.linalg.norm(out - U_ref) <= 1e-9 * np.linalg.norm(U_ref), (pb.kind, pb.nx, pb.ny)
    probe = reqs[0]  # 64^2: the cluster form
    with rd.Batch(1 << 30, 16, small_solve=small) as b:
        pid, pout = b.submit(*probe)
        res = []
        while not res:
            res = b.poll(timeout=5.0)
    assert np.array_equal(pout, ids[0][1]) and res[0]["iterations"] == results[ids[0][0]]["iterations"]


def _requests2():
    """Two-species requests (Gray-Scott periodic, Schnakenberg Neumann, Section 3.4.1) of uneven
    sizes, small ones included (one-launch inner solves)."""
    out = []
    for k, (kind, p, bc, ny, nx, dt) in enumerate([
        ("gray_scott", (2e-3, 1e-3, 0.04, 0.06), "periodic", 64, 64, 1.0),
        ("schnakenberg", (0.05, 1.0, 100.0, 0.1305, 0.7695), "neumann", 128, 128, 1 / 5000),
        ("gray_scott", (2e-3, 1e-3, 0.04, 0.06), "neumann", 256, 128, 1.0),
        ("schnakenberg", (0.05, 1.0, 100.0, 0.1305, 0.7695), "periodic", 8, 8, 1 / 5000),
    ]):
        pb = WL.Problem(nx=nx, ny=ny, lx=1.0, ly=1.0, bc=bc, op="laplacian", kind=kind, p=p, dt=dt,
                        tau_u=0.9, tau_p=0.9, tol=1e-11, tol_kind="f_rel")
        r = WL.rng(110 + k)
        if kind == "gray_scott":
            u0 = np.stack([1 - 0.5 * r.random((ny, nx)), 0.25 * r.random((ny, nx))])
        else:
            u0 = 0.9 + 0.1 * r.random(pb.shape)
        out.append((pb, u0, 3))
    return out


def test_two_species_requests_in_the_batch():
    """Gray-Scott and Schnakenberg requests beside scalar ones: each against the oracle
    (<= 1e-9 rel. L2), and one bit-identical alone and in the mix."""
    reqs = _requests2() + _requests()[:2]
    ids, results, outs, stats = _run(reqs)
    assert len(results) == len(reqs)
    for rid, (pb, u0, n) in zip(ids, reqs):
        r = results[rid]
        assert r["status"] == 0 and r["steps"] == n, r
        U_ref, _ = O.solve(pb, u0, n)
        err = np.linalg.norm(outs[rid] - U_ref) / np.linalg.norm(U_ref)
        assert err <= 1e-9, (pb.kind, pb.bc, pb.ny, pb.nx, err)
    _, res_alone, out_alone, _ = _run([reqs[2]])
    assert np.array_equal(next(iter(out_alone.values())), outs[ids[2]])
    assert next(iter(res_alone.values()))["iterations"] == results[ids[2]]["iterations"]


def test_autotuned_batch_tiles_give_the_same_results():
    """Tiles measured at batch creation (autotune) only change the launch shape: every result
    still agrees with the oracle, and with the fixed-tile batch to the step tolerance."""
    from paper_2305_03945_gb300 import rd
    reqs = _requests()
    outs = {}
    for tune in (0, 1):
        results = {}
        with rd.Batch(1 << 30, 16, autotune=tune) as b:
            ids = [b.submit(pb, u0, n) for pb, u0, n in reqs]
            t0 = time.time()
            while len(results) < len(ids) and time.time() - t0 < 120:
                for r in b.poll(timeout=1.0):
                    results[r["id"]] = r
        assert all(r["status"] == 0 for r in results.values())
        outs[tune] = [o for _, o in ids]
    for (pb, u0, n), a, t in zip(reqs, outs[0], outs[1]):
        U_ref, _ = O.solve(pb, u0, n)
        assert np.linalg.norm(t - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
        assert np.linalg.norm(t - a) <= 1e-9 * np.linalg.norm(U_ref)
