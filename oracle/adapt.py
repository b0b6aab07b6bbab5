"""Adaptive time step size of arxiv 2305.03945, Section 2.2 ("Adaptive time stepsize").

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): imported by tests, never by the product
library.

The paper fixes h_x, tau_u, tau_p and adapts h_t between time steps from the number M of PDHG
iterations the step took, with an upper bound h_t^0, two thresholds N^* > N_* > 0 and a factor
eta in (0, 1):

  * M > N^*             ->  h_t <- eta h_t
  * N_* <= M <= N^*     ->  h_t unchanged
  * M < N_*             ->  h_t <- h_t / eta if h_t / eta <= h_t^0, else unchanged

Readings where the paper is silent:
  * a step whose PDHG solve fails (not converged within max_iter, or diverged) is not accepted:
    it is taken again from U^k with eta h_t (the first rule applied to a step that needed more
    than any N^* iterations);
  * the time loop runs from t = 0 to t_end, and the last step is shortened to end at t_end
    (min(h_t, t_end - t)); the rule acts on the nominal h_t, not on the shortened step;
  * the loop ends when t_end - t <= 1e-12 t_end, or after ``max_attempts`` attempts.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import rd_oracle as O


def next_dt(dt, m, dt0, n_hi, n_lo, eta):
    """The step size after an accepted step that took m PDHG iterations (the three rules)."""
    if m > n_hi:
        return eta * dt
    if m < n_lo:
        up = dt / eta
        return up if up <= dt0 else dt
    return dt


def solve_adaptive(pb, u0, t_end, n_hi, n_lo, eta, max_attempts=1000):
    """Integrate from t = 0 to t_end with h_t^0 = pb.dt.  Returns (U, log, t) where log holds
    one dict per attempt: t (start), dt (used), iterations, status, accepted."""
    dt0 = pb.dt
    dt, t = dt0, 0.0
    U = np.array(u0, dtype=np.float64).reshape(pb.shape)
    log = []
    while t_end - t > 1e-12 * t_end and len(log) < max_attempts:
        h = min(dt, t_end - t)
        Un, info = O.pdhg_step(dataclasses.replace(pb, dt=h), U)
        ok = info["status"] == O.OK
        log.append({"t": t, "dt": h, "iterations": info["iterations"], "status": info["status"],
                    "accepted": ok})
        if ok:
            U = Un
            t = t + h
            dt = next_dt(dt, info["iterations"], dt0, n_hi, n_lo, eta)
        else:
            dt = eta * dt
    return U, log, t


def replay(pb, u0, dts):
    """Fixed steps of the given sizes from u0 (the accepted steps of an adaptive run)."""
    U = np.array(u0, dtype=np.float64).reshape(pb.shape)
    infos = []
    for h in dts:
        U, info = O.pdhg_step(dataclasses.replace(pb, dt=h), U)
        infos.append(info)
    return U, infos
