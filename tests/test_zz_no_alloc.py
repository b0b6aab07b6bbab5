"""The allocation-free preconditioner solve (rd_apply_precond_static) against the handle-based
one (rd_pdhg_apply_precond), through the C ABI, on two calls in a row (and, on the same inputs,
against the oracle's G^{-1}).

This entry point serves callers that cannot allocate device memory when they need G^{-1} W
(a fixed memory budget they do not own, loops that must not pay cudaMalloc's device-wide
synchronisation, or no solver handle at hand): its scratch lives in a static device array
shared by all calls.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from oracle import rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("allen_cahn", "laplacian", (), "periodic", (64, 64)),
    ("allen_cahn", "laplacian", (), "neumann", (32, 128)),
    ("ch_implicit", "neg_biharmonic", (), "periodic", (128, 64)),
    ("ch_split", "neg_biharmonic", (), "neumann", (64, 64)),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06), "periodic", (128, 128)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695), "neumann", (256, 256)),
    # the longest lines the static solve admits (side 2048): row lines of 2048 points, column
    # lines of 2048 points, and a two-row grid of 2048-point rows
    ("allen_cahn", "laplacian", (), "periodic", (64, 2048)),
    ("allen_cahn", "laplacian", (), "neumann", (64, 2048)),
    ("allen_cahn", "laplacian", (), "periodic", (2048, 64)),
    ("allen_cahn", "laplacian", (), "neumann", (2048, 64)),
    ("ch_split", "neg_biharmonic", (), "neumann", (2, 2048)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2305_03945_gb300 import build
    build.build()


def _pb(kind, op, p, bc, ny, nx):
    ch = op == "neg_biharmonic"
    return WL.Problem(nx=nx, ny=ny, lx=1.0, ly=1.3, bc=bc, op=op, kind=kind, p=p,
                      dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0)


def _static(pb, w, y):
    from paper_2305_03945_gb300 import rd
    lib = rd.load()
    g, rx, pc, o = rd.make_structs(pb)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.rd_apply_precond_static(ctypes.byref(g), rd.BC[pb.bc], rd.OP[pb.op], ctypes.byref(rx), pb.dt,
                                       ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                       ctypes.c_void_p(stream))


@pytest.mark.parametrize("kind,op,p,bc,shape", CASES)
def test_static_scratch_solve_matches_handle_solve_twice(kind, op, p, bc, shape):
    from paper_2305_03945_gb300 import rd
    pb = _pb(kind, op, p, bc, *shape)
    with rd.Solver(pb) as s:
        for call in range(2):  # two calls in a row share (and reuse) the static scratch
            W = torch.from_numpy(WL.rng(100 + call).standard_normal(pb.shape)).cuda()
            want = torch.empty_like(W)
            s.apply_precond(W, want)
            got = torch.empty_like(W)
            assert _static(pb, W, got) == rd.RD_OK, rd.load().rd_last_error()
            torch.cuda.synchronize()
            g, t = got.cpu().numpy(), want.cpu().numpy()
            assert np.max(np.abs(g - t)) <= 1e-12 * np.max(np.abs(t))
            # and directly against the oracle's FFT / DCT solve of the same G
            ref = O.apply_ginv(pb, W.cpu().numpy())
            assert np.max(np.abs(g - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_static_scratch_rejects_grids_beyond_its_limit():
    from paper_2305_03945_gb300 import rd
    pb = _pb("allen_cahn", "laplacian", (), "periodic", 512, 512)  # 262144 points > 131072
    W = torch.zeros(pb.shape, dtype=torch.float64, device="cuda")
    assert _static(pb, W, W) == rd.RD_ERR_UNSUPPORTED
    assert b"131072" in rd.load().rd_last_error()


@pytest.mark.parametrize("ny,nx", [(2, 4096), (4096, 2)])
def test_static_scratch_rejects_sides_beyond_2048(ny, nx):
    from paper_2305_03945_gb300 import rd
    pb = _pb("allen_cahn", "laplacian", (), "neumann", ny, nx)  # 8192 points: within the point limit
    W = torch.zeros(pb.shape, dtype=torch.float64, device="cuda")
    assert _static(pb, W, W) == rd.RD_ERR_UNSUPPORTED
    assert b"2048" in rd.load().rd_last_error()
