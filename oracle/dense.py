"""Dense-matrix forms of the implicit step, for pinning the oracle on tiny grids.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The Laplacians are written out entry by entry from the block forms the paper prints:
  Lap^P  (Section 2.1): block-circulant, diagonal blocks L = circ(-4, 1, ..., 1), off-diagonal
         and corner blocks I, all over h^2;
  Lap^N  (Remark 1, eq. def Lap N): block-tridiagonal, diagonal blocks L_1 (first and last block
         rows; diagonal -2, -3, ..., -3, -2) and L_2 (interior; diagonal -3, -4, ..., -4, -3),
         off-diagonal blocks I, all over h^2.
Vectorisation l = i*N + j (i the block / y index, j the x index), as in Section 2.1.
The residual, Jacobian and Newton solve below use only these dense matrices and pointwise
formulas, so they share no stencil or transform code with ``rd_oracle``.
"""
from __future__ import annotations

import numpy as np


def _tridiag(n, diag):
    m = np.zeros((n, n))
    for j in range(n):
        m[j, j] = diag[j]
        if j + 1 < n:
            m[j, j + 1] = 1.0
            m[j + 1, j] = 1.0
    return m


def lap_periodic(n, h):
    """Lap^P for an n x n periodic grid (n >= 3 so that the corner entries are distinct)."""
    assert n >= 3
    L = _tridiag(n, [-4.0] * n)
    L[0, n - 1] = 1.0
    L[n - 1, 0] = 1.0
    I = np.eye(n)
    M = np.zeros((n * n, n * n))
    for bi in range(n):
        M[bi * n:(bi + 1) * n, bi * n:(bi + 1) * n] = L
        for bj in ((bi + 1) % n, (bi - 1) % n):
            M[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n] = I
    return M / h ** 2


def lap_neumann(n, h):
    """Lap^N for an n x n grid with the half-cell mirror ghost (n >= 3)."""
    assert n >= 3
    L1 = _tridiag(n, [-2.0] + [-3.0] * (n - 2) + [-2.0])
    L2 = _tridiag(n, [-3.0] + [-4.0] * (n - 2) + [-3.0])
    I = np.eye(n)
    M = np.zeros((n * n, n * n))
    for bi in range(n):
        M[bi * n:(bi + 1) * n, bi * n:(bi + 1) * n] = L1 if bi in (0, n - 1) else L2
        for bj in (bi + 1, bi - 1):
            if 0 <= bj < n:
                M[bi * n:(bi + 1) * n, bj * n:(bj + 1) * n] = I
    return M / h ** 2


def second_difference(n, h, bc):
    """1-D second difference (x_{j+1} + x_{j-1} - 2 x_j) / h^2 on n points: circulant (periodic)
    or with the half-cell mirror ghost x_{-1} = x_0, x_n = x_{n-1} (Neumann, Remark 1)."""
    m = np.zeros((n, n))
    for j in range(n):
        m[j, j] -= 2.0
        for k in (j - 1, j + 1):
            if 0 <= k < n:
                m[j, k] += 1.0
            elif bc == "periodic":
                m[j, k % n] += 1.0
            else:
                m[j, j] += 1.0
    return m / h ** 2


def lap_kron(pb):
    """Lap as the Kronecker sum of the 1-D second differences, vectorised l = (z ny + y) nx + x:
    I_z (x) I_y (x) D_x + I_z (x) D_y (x) I_x [+ D_z (x) I_y (x) I_x on 3-D grids]."""
    Dx = second_difference(pb.nx, pb.lx / pb.nx, pb.bc)
    Dy = second_difference(pb.ny, pb.ly / pb.ny, pb.bc)
    Ix, Iy = np.eye(pb.nx), np.eye(pb.ny)
    L = np.kron(Iy, Dx) + np.kron(Dy, Ix)
    if pb.nz > 1:
        Dz = second_difference(pb.nz, pb.lz / pb.nz, pb.bc)
        Iz = np.eye(pb.nz)
        L = np.kron(Iz, L) + np.kron(Dz, np.kron(Iy, Ix))
    return L


def lap_matrix(pb):
    """The paper's block matrices Lap^P / Lap^N on square 2-D grids; the Kronecker-sum form on
    3-D grids (the paper prints no 3-D matrix)."""
    if pb.nz > 1:
        return lap_kron(pb)
    assert pb.nx == pb.ny and abs(pb.lx - pb.ly) < 1e-15, "dense pins use square grids"
    h = pb.lx / pb.nx
    return lap_periodic(pb.nx, h) if pb.bc == "periodic" else lap_neumann(pb.nx, h)


def linear_part(pb, L=None):
    """Per-component dense A_lin (list): I - D dt Lap, or I + a dt Lap^2."""
    L = lap_matrix(pb) if L is None else L
    I = np.eye(L.shape[0])
    if pb.kind in ("gray_scott", "schnakenberg"):
        return [I - pb.p[0] * pb.dt * L, I - pb.p[1] * pb.dt * L]
    if pb.op == "laplacian":
        return [I - pb.a * pb.dt * L]
    if pb.op == "functionalized":   # I - dt Lap (a Lap - (2b - a) I) a Lap (Section 3.3's G root)
        return [I - pb.dt * L @ (pb.a * L - (2 * pb.b - pb.a) * I) @ (pb.a * L)]
    return [I + pb.a * pb.dt * (L @ L)]


def residual(pb, U, Uk, L=None):
    """F(U) with dense matrices; U, Uk flat vectors of length ncomp*N^2."""
    L = lap_matrix(pb) if L is None else L
    N2 = L.shape[0]
    dt, a, b = pb.dt, pb.a, pb.b
    if pb.ncomp == 1:
        A = linear_part(pb, L)[0]
        if pb.kind == "none":
            return A @ U - Uk
        if pb.kind == "allen_cahn":
            return A @ U - Uk + dt * b * (U ** 3 - U)
        if pb.kind == "ch_implicit":
            return A @ U - Uk - dt * b * (L @ (U ** 3 - U))
        if pb.kind == "ch_split":
            return A @ U - Uk - dt * b * (L @ U ** 3) + dt * b * (L @ Uk)
        if pb.kind == "fch":        # U - U^k - dt Lap (a Lap - b W'' + a)(a Lap U - b W')
            I = np.eye(N2)
            mu = a * (L @ U) - b * (U ** 3 - U)
            Am = (a * L - b * np.diag(3 * U ** 2 - 1) + a * I) @ mu
            return U - Uk - dt * (L @ Am)
    u, v = U[:N2], U[N2:]
    uk, vk = Uk[:N2], Uk[N2:]
    Au, Av = linear_part(pb, L)
    if pb.kind == "gray_scott":
        Du, Dv, Ff, k = pb.p
        Fu = Au @ u - uk + dt * (u * v * v) - dt * Ff * (1 - u)
        Fv = Av @ v - vk - dt * (u * v * v) + dt * (Ff + k) * v
        return np.concatenate([Fu, Fv])
    if pb.kind == "schnakenberg":
        D1, D2, kap, a_s, b_s = pb.p
        Fu = Au @ u - uk - dt * kap * (a_s - u + u * u * v)
        Fv = Av @ v - vk - dt * kap * (b_s - u * u * v)
        return np.concatenate([Fu, Fv])
    raise ValueError(pb.kind)


def jacobian(pb, U, L=None):
    """Dense dF/dU, assembled from the linear part and the pointwise derivatives."""
    L = lap_matrix(pb) if L is None else L
    N2 = L.shape[0]
    dt, b = pb.dt, pb.b
    if pb.ncomp == 1:
        A = linear_part(pb, L)[0]
        if pb.kind == "none":
            return A
        if pb.kind == "allen_cahn":
            return A + np.diag(dt * b * (3 * U ** 2 - 1))
        if pb.kind == "ch_implicit":
            return A - dt * b * L @ np.diag(3 * U ** 2 - 1)
        if pb.kind == "ch_split":
            return A - dt * b * L @ np.diag(3 * U ** 2)
        if pb.kind == "fch":        # product rule on Lap A(U) mu(U)
            a = pb.a
            I = np.eye(N2)
            mu = a * (L @ U) - b * (U ** 3 - U)
            Amat = a * L - b * np.diag(3 * U ** 2 - 1) + a * I
            Bmat = a * L - b * np.diag(3 * U ** 2 - 1)
            return I - dt * L @ (Amat @ Bmat - b * np.diag(6 * U * mu))
    u, v = U[:N2], U[N2:]
    Au, Av = linear_part(pb, L)
    if pb.kind == "gray_scott":
        Du, Dv, Ff, k = pb.p
        Juu = Au + np.diag(dt * (v * v + Ff))
        Juv = np.diag(2 * dt * u * v)
        Jvu = np.diag(-dt * v * v)
        Jvv = Av + np.diag(-dt * (2 * u * v - (Ff + k)))
    else:
        D1, D2, kap, a_s, b_s = pb.p
        Juu = Au - np.diag(dt * kap * (-1 + 2 * u * v))
        Juv = np.diag(-dt * kap * u * u)
        Jvu = np.diag(2 * dt * kap * u * v)
        Jvv = Av + np.diag(dt * kap * u * u)
    return np.block([[Juu, Juv], [Jvu, Jvv]])


def newton(pb, Uk, tol=1e-14, max_iter=50):
    """Dense Newton with LU (numpy.linalg.solve) from U = U^k until ||F||_2 <= tol * max(1,||U^k||)."""
    L = lap_matrix(pb)
    Uk = np.asarray(Uk, dtype=np.float64).ravel()
    U = Uk.copy()
    for _ in range(max_iter):
        Fv = residual(pb, U, Uk, L)
        if np.linalg.norm(Fv) <= tol * max(1.0, np.linalg.norm(Uk)):
            return U.reshape(pb.shape)
        U = U - np.linalg.solve(jacobian(pb, U, L), Fv)
    raise RuntimeError("dense Newton did not converge")


def preconditioner(pb):
    """Dense block-diagonal G = diag(A_lin,c^2)."""
    As = linear_part(pb)
    n = As[0].shape[0]
    G = np.zeros((n * len(As), n * len(As)))
    for c, A in enumerate(As):
        G[c * n:(c + 1) * n, c * n:(c + 1) * n] = A @ A
    return G
