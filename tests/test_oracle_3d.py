"""Pins of the oracles' 3-D grids, CPU only.

The paper is 2-D; a 3-D grid is its scheme with a third axis (seven-point Laplacian, the symbol
with a third sin^2 term, transforms along all three axes).  Each piece is pinned from outside the
oracle code: the Laplacian against the dense Kronecker sum of 1-D second differences (itself
checked against the paper's 2-D block matrices), eigenmodes against the closed-form symbol, G^{-1}
against a dense solve, the reaction-off step against the closed-form decay, the nonlinear step
against dense Newton, and Cahn-Hilliard mass conservation.  Every test runs against both oracles.
"""
import math

import numpy as np
import pytest

from oracle import cpp_oracle, dense as D, rd_oracle
from paper_2305_03945_gb300 import workloads as WL


@pytest.fixture(params=["numpy", "cpp"])
def O(request):
    if request.param == "cpp":
        cpp_oracle.set_threads(1)
        yield cpp_oracle
        cpp_oracle.set_threads(0)
    else:
        yield rd_oracle


def _pb(bc, nz, ny, nx, kind="none", op="laplacian", **kw):
    ch = op == "neg_biharmonic"
    base = dict(nx=nx, ny=ny, nz=nz, lx=1.0, ly=0.8, lz=1.3, bc=bc, op=op, kind=kind,
                dt=1e-5 if ch else 2e-3, a=4e-4 if ch else 0.05, b=1.0 if ch else 20.0,
                tau_u=0.9, tau_p=0.9, tol=1e-13, tol_kind="f_rel", max_iter=20000)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("n", [3, 4, 5])
def test_kron_laplacian_is_the_paper_block_matrix_in_2d(bc, n):
    pb = WL.Problem(nx=n, ny=n, lx=1.0, ly=1.0, bc=bc, op="laplacian", kind="none", dt=1.0)
    h = 1.0 / n
    want = D.lap_periodic(n, h) if bc == "periodic" else D.lap_neumann(n, h)
    assert np.allclose(D.lap_kron(pb), want, rtol=0, atol=1e-12 / h ** 2)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("shape", [(3, 4, 5), (4, 4, 4), (2, 8, 4)])
def test_seven_point_laplacian_is_the_kron_sum(bc, shape, O):
    pb = _pb(bc, *shape)
    u = WL.rng(11).standard_normal(pb.shape)
    W = O.residual(pb, u, np.zeros(pb.shape))        # (I - a dt Lap) u
    lap = (u - W) / (pb.a * pb.dt)
    want = (D.lap_kron(pb) @ u.ravel()).reshape(pb.shape)
    assert np.max(np.abs(lap - want)) <= 1e-9 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("k", [(1, 0, 2), (3, 2, 1), (0, 5, 7)])
def test_3d_eigenmodes_and_symbol(bc, k, O):
    pb = _pb(bc, 8, 8, 16)
    kz, ky, kx = k
    z = np.arange(pb.nz)[:, None, None]
    y = np.arange(pb.ny)[None, :, None]
    x = np.arange(pb.nx)[None, None, :]
    if bc == "periodic":
        phi = np.cos(2 * np.pi * (kx * x / pb.nx + ky * y / pb.ny + kz * z / pb.nz))
        d = 1
    else:
        phi = (np.cos(np.pi * kx * (x + 0.5) / pb.nx) * np.cos(np.pi * ky * (y + 0.5) / pb.ny)
               * np.cos(np.pi * kz * (z + 0.5) / pb.nz))
        d = 2
    mu = sum(4 / h ** 2 * math.sin(math.pi * kk / (d * n)) ** 2
             for kk, n, h in ((kx, pb.nx, pb.lx / pb.nx), (ky, pb.ny, pb.ly / pb.ny), (kz, pb.nz, pb.lz / pb.nz)))
    W = O.residual(pb, phi[None], np.zeros(pb.shape))
    assert np.max(np.abs(W[0] - (1 + pb.a * pb.dt * mu) * phi)) <= 1e-12 * (1 + pb.a * pb.dt * mu)
    g = O.ghat(pb)[0]
    idx = (kz, ky, kx)
    assert g[idx] == pytest.approx((1 + pb.a * pb.dt * mu) ** 2, rel=1e-13)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", [("allen_cahn", "laplacian", ()), ("ch_split", "neg_biharmonic", ()),
                                       ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06))])
def test_3d_ginv_matches_dense_solve(bc, kind, op, p, O):
    pb = _pb(bc, 4, 4, 8, kind=kind, op=op, p=p)
    W = WL.rng(12).standard_normal(pb.shape)
    got = O.apply_ginv(pb, W)
    want = np.linalg.solve(D.preconditioner(pb), W.ravel()).reshape(pb.shape)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_3d_reaction_off_mode_decays_at_closed_form_rate(bc, O):
    pb = _pb(bc, 8, 4, 8, tau_u=1.0, tau_p=1.0)
    x = np.arange(pb.nx)[None, None, :]
    z = np.arange(pb.nz)[:, None, None]
    if bc == "periodic":
        phi, d = np.cos(2 * np.pi * (2 * x / pb.nx + 3 * z / pb.nz)) + 0 * np.arange(pb.ny)[None, :, None], 1
    else:
        phi = np.cos(np.pi * 2 * (x + 0.5) / pb.nx) * np.cos(np.pi * 3 * (z + 0.5) / pb.nz) + 0 * np.arange(pb.ny)[None, :, None]
        d = 2
    mu = 4 / (pb.lx / pb.nx) ** 2 * math.sin(math.pi * 2 / (d * pb.nx)) ** 2 + \
        4 / (pb.lz / pb.nz) ** 2 * math.sin(math.pi * 3 / (d * pb.nz)) ** 2
    U, infos = O.solve(pb, phi[None], 5)
    assert all(i["status"] == "ok" for i in infos)
    assert np.max(np.abs(U[0] - phi * (1 + pb.dt * pb.a * mu) ** -5)) <= 1e-12


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_3d_unit_steps_are_nilpotent(bc, O):
    pb = _pb(bc, 4, 8, 4, tau_u=1.0, tau_p=1.0)
    uk = WL.rng(13).standard_normal(pb.shape)
    U, info = O.pdhg_step(pb, uk)
    assert info["status"] == "ok" and info["iterations"] == 2


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", [("allen_cahn", "laplacian", ()), ("ch_split", "neg_biharmonic", ()),
                                       ("ch_implicit", "neg_biharmonic", ()),
                                       ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06))])
def test_3d_nonlinear_step_matches_dense_newton(bc, kind, op, p, O):
    pb = _pb(bc, 4, 4, 4, kind=kind, op=op, p=p)
    r = WL.rng(14)
    uk = np.abs(r.uniform(0.2, 0.8, pb.shape)) if kind == "gray_scott" else r.uniform(-0.8, 0.8, pb.shape)
    U, info = O.pdhg_step(pb, uk)
    assert info["status"] == "ok"
    Un = D.newton(pb, uk)
    assert np.max(np.abs(U - Un)) <= 1e-10 * np.max(np.abs(Un))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind", ["ch_implicit", "ch_split"])
def test_3d_cahn_hilliard_conserves_mass(bc, kind, O):
    pb = _pb(bc, 8, 8, 8, kind=kind, op="neg_biharmonic", tol=1e-12)
    u0 = WL.zero_mean_uniform(15, pb.shape, 0.3) + 0.1
    U, infos = O.solve(pb, u0, 3)
    assert all(i["status"] == "ok" for i in infos)
    h3 = (pb.lx / pb.nx) * (pb.ly / pb.ny) * (pb.lz / pb.nz)
    assert abs(h3 * (U.sum() - u0.sum())) <= 1e-12
