"""A second, independent solver of the same implicit Cahn-Hilliard step, for long runs.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The fully implicit periodic Cahn-Hilliard step of eq. (F(U) CH) (sign reading lambda = -a),

    F(U) = (I + a dt Lap^2) U - U^k - b dt Lap (U^3 - U) = 0,

is solved here not by PDHG but by a stabilised fixed point in the Fourier basis of the periodic
five-point Laplacian (-Lap has the symbol mu of ``rd_oracle.symbol_mu``): with a constant S > 0,

    (1 + a dt mu^2 + S b dt mu) U_{m+1}^ = U^k^ - b dt mu (U_m^3 - U_m)^ + S b dt mu U_m^ ,

whose fixed points are exactly the roots of F.  A run of thousands of steps on a 128^2 grid
takes minutes this way instead of hours with the PDHG oracle, and the two solvers share nothing
but the residual map F, which the solution is checked against.
"""
from __future__ import annotations

import numpy as np

from . import rd_oracle as O


def ch_implicit_step(pb, Uk, S=2.0, tol=1e-14, max_iter=500):
    """One implicit step for pb.kind == 'ch_implicit', pb.bc == 'periodic'.  Returns (U, its)."""
    assert pb.kind == "ch_implicit" and pb.bc == "periodic" and pb.ncomp == 1
    mu = O.symbol_mu(pb)
    dt, a, b = pb.dt, pb.a, pb.b
    den = 1.0 + a * dt * mu ** 2 + S * b * dt * mu
    uk = np.asarray(Uk, dtype=np.float64)[0]
    ukh = np.fft.fft2(uk)
    u = uk.copy()
    for m in range(1, max_iter + 1):
        rhs = ukh - b * dt * mu * np.fft.fft2(u ** 3 - u) + S * b * dt * mu * np.fft.fft2(u)
        un = np.real(np.fft.ifft2(rhs / den))
        d = float(np.max(np.abs(un - u)))
        u = un
        if d <= tol:
            return u[None], m
    raise RuntimeError("fixed point did not converge in %d iterations" % max_iter)


def sign_change_steps(pb, u0, points, nsteps):
    """Run nsteps implicit steps from u0 and return, for each grid point (j, i), the first step
    after which U[0, j, i] has the opposite sign of u0 there (None if it never changes)."""
    U = np.asarray(u0, dtype=np.float64)
    s0 = [np.sign(U[0, j, i]) for j, i in points]
    out = [None] * len(points)
    for k in range(1, nsteps + 1):
        U, _ = ch_implicit_step(pb, U)
        for q, (j, i) in enumerate(points):
            if out[q] is None and np.sign(U[0, j, i]) != s0[q]:
                out[q] = k
        if all(o is not None for o in out):
            break
    return out
