"""Pins of the oracle's grid operators, transforms and preconditioner (CPU only).

Each test checks ``oracle.rd_oracle`` against something other than itself: the dense block
matrices printed in the paper, textbook eigenvalues, brute-force transform definitions and
dense linear solves.
"""
import numpy as np
import pytest

from oracle import dense, rd_oracle as O
from paper_2305_03945_gb300 import workloads as WL


def _pb(n=8, bc="periodic", op="laplacian", kind="none", **kw):
    base = dict(nx=n, ny=n, lx=1.0, ly=1.0, bc=bc, op=op, kind=kind, dt=1e-3, a=0.5, b=2.0)
    base.update(kw)
    return WL.Problem(**base)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("n", [3, 4, 5, 8])
def test_stencil_equals_paper_block_matrix(bc, n):
    """Lap^P (Section 2.1) and Lap^N (Remark 1) written out entry by entry equal the stencil."""
    pb = _pb(n, bc)
    u = WL.rng(n).standard_normal((1, n, n))
    M = dense.lap_matrix(pb)
    got = O.lap(u, pb)[0].ravel()
    want = M @ u[0].ravel()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_neumann_block_diagonals_as_printed():
    """The printed L_1 / L_2 diagonals: corners -2, edges -3, interior -4 (times 1/h^2)."""
    M = dense.lap_neumann(4, 1.0)
    diag = np.diag(M).reshape(4, 4)
    assert diag[0].tolist() == [-2, -3, -3, -2]
    assert diag[1].tolist() == [-3, -4, -4, -3]
    assert np.allclose(M, M.T)
    assert np.allclose(M.sum(axis=1), 0)          # mirror ghost: rows sum to zero


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("shape", [(16, 16), (8, 32)])
@pytest.mark.parametrize("k", [(0, 1), (3, 2), (5, 7)])
def test_stencil_eigenmodes(bc, shape, k):
    """The five-point Laplacian maps a Fourier (periodic) or DCT-II (Neumann) mode to
    -mu times itself, mu = 4/h^2 sin^2(pi k / N) per axis (periodic, Section 2.1 after
    Theorem 1) or 4/h^2 sin^2(pi k / (2N)) (Neumann, cosine basis of Remark 1)."""
    ny, nx = shape
    pb = _pb(bc=bc, nx=nx, ny=ny, lx=2.0, ly=1.5)
    kx, ky = k[0] % nx, k[1] % ny
    m = WL.cosine_mode(pb, kx, ky)
    hx, hy = 2.0 / nx, 1.5 / ny
    d = 1 if bc == "periodic" else 2
    mu = 4 / hx ** 2 * np.sin(np.pi * kx / (d * nx)) ** 2 + 4 / hy ** 2 * np.sin(np.pi * ky / (d * ny)) ** 2
    got = O.lap(m, pb)
    assert np.max(np.abs(got + mu * m)) <= 1e-12 * max(1.0, mu)


def test_periodic_heat_condition_number_matches_paper():
    """Section 2.1: eigenvalues of I - h_t lam Lap^P are 1 + 4 h_t lam N^2 sin^2(pi k/N) on a
    unit 1-D grid, so kappa = 1 + 4 lam N^2 h_t for even N.  On the 2-D grid the same
    statement holds per axis; the x-only modes (ky = 0) reproduce the 1-D spectrum."""
    n, lam, ht = 16, 0.3, 2e-3
    pb = _pb(n, "periodic", dt=ht, a=lam)
    A = np.eye(n * n) - ht * lam * dense.lap_matrix(pb)
    ev = np.linalg.eigvalsh(A)
    k = np.arange(n)
    one_d = 1 + 4 * ht * lam * n ** 2 * np.sin(np.pi * k / n) ** 2
    # the 2-D spectrum is the set of sums of two 1-D spectra minus 1
    two_d = np.sort((one_d[:, None] + one_d[None, :] - 1).ravel())
    assert np.allclose(np.sort(ev), two_d, rtol=1e-12)
    assert abs(one_d.max() / one_d.min() - (1 + 4 * lam * n ** 2 * ht)) < 1e-12


def _dct2_brute(x):
    n = len(x)
    j = np.arange(n)
    return np.array([np.sum(x * np.cos(np.pi * k * (2 * j + 1) / (2 * n))) for k in range(n)])


def test_oracle_neumann_basis_is_dct2():
    """The oracle's Neumann transform is the DCT-II (Remark 1): compare its orthonormal
    coefficients with the brute-force definition X_k = sum_j x_j cos(pi k (2j+1)/(2N))."""
    import scipy.fft as sfft
    x = WL.rng(5).standard_normal(16)
    X = _dct2_brute(x)
    scale = np.sqrt(2 / 16) * np.where(np.arange(16) == 0, np.sqrt(0.5), 1.0)
    assert np.allclose(sfft.dct(x, type=2, norm="ortho"), scale * X, atol=1e-13)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", [
    ("none", "laplacian", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
    ("fch", "functionalized", ()),
])
def test_ginv_matches_dense_solve(bc, kind, op, p):
    """G^{-1} W through the spectral symbol equals a dense Cholesky solve with
    G = A_lin^2 assembled from the paper's dense Laplacian."""
    import scipy.linalg as sla
    dt = {"laplacian": 2e-3, "neg_biharmonic": 1e-5, "functionalized": 1e-8}[op]
    pb = _pb(16, bc, op=op, kind=kind, p=p, dt=dt, a=0.2)
    W = WL.rng(11).standard_normal(pb.shape)
    got = O.apply_ginv(pb, W).ravel()
    G = dense.preconditioner(pb)
    want = sla.cho_solve(sla.cho_factor(G), W.ravel())
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", [
    ("none", "laplacian", ()),
    ("none", "neg_biharmonic", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("ch_split", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
    ("fch", "functionalized", ()),
])
def test_residual_matches_dense_form(bc, kind, op, p):
    """The stencil-based F(U) equals F written with the paper's dense matrices."""
    pb = _pb(8, bc, op=op, kind=kind, p=p, dt=3e-3, a=0.1, b=1.5)
    r = WL.rng(3)
    U = r.uniform(-1, 1, pb.shape)
    Uk = r.uniform(-1, 1, pb.shape)
    got = O.residual(pb, U, Uk).ravel()
    want = dense.residual(pb, U.ravel(), Uk.ravel())
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("kind,op,p", [
    ("none", "laplacian", ()),
    ("none", "neg_biharmonic", ()),
    ("allen_cahn", "laplacian", ()),
    ("ch_implicit", "neg_biharmonic", ()),
    ("ch_split", "neg_biharmonic", ()),
    ("gray_scott", "laplacian", (2e-3, 1e-3, 0.04, 0.06)),
    ("schnakenberg", "laplacian", (0.05, 1.0, 100.0, 0.1305, 0.7695)),
    ("fch", "functionalized", ()),
])
def test_adjoint_jacobian_by_complex_step(bc, kind, op, p):
    """<grad_F_T(U) P, V> = <P, J V> with J V from the complex-step derivative of F
    (exact to rounding for these polynomial F): pins the U-update of the dynamic."""
    pb = _pb(8, bc, op=op, kind=kind, p=p, dt=3e-3, a=0.1, b=1.5)
    r = WL.rng(4)
    U = r.uniform(-1, 1, pb.shape)
    Uk = r.uniform(-1, 1, pb.shape)
    P = r.standard_normal(pb.shape)
    V = r.standard_normal(pb.shape)
    h = 1e-30
    JV = np.imag(O.residual(pb, U + 1j * h * V, Uk.astype(complex))) / h
    lhs = np.sum(O.grad_F_T(pb, U, P) * V)
    rhs = np.sum(P * JV)
    assert abs(lhs - rhs) <= 1e-12 * (abs(rhs) + np.sum(np.abs(P * JV)))
    # and against the dense Jacobian
    J = dense.jacobian(pb, U.ravel())
    assert np.allclose(J @ V.ravel(), JV.ravel(), rtol=1e-12, atol=1e-12)
    assert np.allclose(J.T @ P.ravel(), O.grad_F_T(pb, U, P).ravel(), rtol=1e-12, atol=1e-12)


def test_ginv_spectrum_positive_for_ch_sign_reading():
    """With F = (I + a dt Lap^2) U - ..., G = (I + a dt Lap^2)^2 is SPD with smallest
    eigenvalue exactly 1 (the constant mode)."""
    pb = _pb(16, "periodic", op="neg_biharmonic", kind="ch_implicit", dt=1e-5, a=4e-4)
    g = O.ghat(pb)
    assert g.min() == 1.0 and np.all(g >= 1.0)
