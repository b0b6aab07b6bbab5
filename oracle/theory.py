"""Closed forms of the linear convergence analysis (Theorem 1, Corollary 1, Appendix A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import math

import numpy as np


def iteration_matrix(tau_u, tau_p, lam, omega=1.0):
    """Per-eigenmode PDHG matrix D_k of Appendix A for F(U) = A U - b with A symmetric:
    error e and dual p evolve as p' = p + tau_p lam e, e' = e - tau_u lam (p + (1+omega) tau_p lam e).
    For omega = 1 this is [[1 - 2 tau_u tau_p lam^2, -tau_u lam], [tau_p lam, 1]]."""
    t = tau_u * tau_p * lam * lam
    return np.array([[1 - (1 + omega) * t, -tau_u * lam], [tau_p * lam, 1.0]])


def rate(t):
    """Spectral radius f(t) of D_k as a function of t = tau_u tau_p lam^2 (Appendix A)."""
    if t <= 1:
        return math.sqrt(1 - t)
    return t - 1 + math.sqrt(t * t - t)


def _bracket(kappa):
    k2 = kappa * kappa
    return (0.75 * k2 + 1.5 - 0.25 / k2
            + (kappa - 1) / (2 * kappa) * math.sqrt((kappa - 1) * (3 * kappa + 1))
            * math.sqrt(0.75 * k2 + 1.5 + 2 * kappa - 0.25 / k2))


def eta_star(kappa):
    """Optimal eta = tau_u tau_p lam_max^2 (Remark 2, explicit formula)."""
    return 2 * kappa * kappa / _bracket(kappa)


def gamma_star(kappa):
    """Optimal rate gamma_* (Remark 2, explicit formula)."""
    return math.sqrt(1 - 2 / _bracket(kappa))


def single_mode_residuals(alpha, g, tau_u, tau_p, omega, e0, n_iter):
    """Residual coefficients alpha*e_n of the G-prox dynamic restricted to one eigenmode.

    For F(U) = A U - U^k with A alpha on the mode and G g on the mode:
      p_{n+1} = p_n + tau_p (alpha/g) e_n
      e_{n+1} = e_n - tau_u alpha (p_n + (1+omega) tau_p (alpha/g) e_n)
    (eqs. G-prox linearized pdhg dynamic 1-3 applied to a single eigenvector).
    """
    e, p = e0, 0.0
    out = [alpha * e]
    for _ in range(n_iter):
        y = alpha * e / g
        pt = p + (1 + omega) * tau_p * y
        p = p + tau_p * y
        e = e - tau_u * alpha * pt
        out.append(alpha * e)
    return np.array(out)
