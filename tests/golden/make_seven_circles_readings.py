"""Write seven_circles_readings.json: the zero-crossing times of the seven-circle example of
Section 3.2.1 (Table 1) under each alternative reading of its set-up, to see which, if any, gives
the printed T1 in [6.340, 6.345] and T2 in [26.015, 26.020].

Each reading changes one thing against the baseline (a = 0.1^2, b = 1 with W = (u^2 - 1)^2 / 4,
N_x = 128 periodic nodes at j h, h_t = 1/200, mollifier eps = 0.1, five-point Laplacian):

  cell_centres    nodes at (j + 1/2) h; u at (pi/2, pi/2) read by bilinear interpolation
  w_unscaled      W = (u^2 - 1)^2, i.e. W' = 4 (u^3 - u): b = 4
  a_0.1           a = 0.1 instead of 0.1^2
  mollifier_0.05  mollifier eps = 0.05 (a sharper initial profile)
  dt_1/800        h_t = 1/800 (time refinement of the same scheme)
  n_256           N_x = 256, h = pi/128 (space refinement)

Calls only ``oracle/`` (the fixed-point implicit step of oracle/fixed_point.py, which solves
F(U) = 0 of the PDHG oracle to max |dU| <= 1e-14) and the seeded-input module.  The readings run
in parallel processes; the slowest (dt_1/800, n_256) take about forty minutes.

    python tests/golden/make_seven_circles_readings.py [reading ...]
"""
import dataclasses
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fixed_point as FP  # noqa: E402
from paper_2305_03945_gb300 import workloads as WL  # noqa: E402

READINGS = ("baseline", "cell_centres", "w_unscaled", "a_0.1", "mollifier_0.05", "dt_1/800", "n_256")
T_END = 30.0


def setup(name):
    """(problem, u0, probe) of one reading; probe(U) -> (u at (pi/2, pi/2), u at (3pi/2, 3pi/2))."""
    n = 256 if name == "n_256" else 128
    w = WL.config_seven_circles(n)
    pb = w.problem
    off = 0.5 if name == "cell_centres" else 0.0
    eps = 0.05 if name == "mollifier_0.05" else 0.1
    u0 = WL.seven_circles(n, node_offset=off, mollifier_eps=eps)
    if name == "w_unscaled":
        pb = dataclasses.replace(pb, b=4.0)
    if name == "a_0.1":
        pb = dataclasses.replace(pb, a=0.1)
    if name == "dt_1/800":
        pb = dataclasses.replace(pb, dt=1 / 800)
    q1, q3 = n // 4, 3 * n // 4          # pi/2 and 3pi/2 are nodes q h (h = 2 pi / n)

    def probe(U):
        u = U[0]
        if off == 0.0:
            return float(u[q1, q1]), float(u[q3, q3])
        # cell centres (j + 1/2) h: the point q h sits midway between nodes q - 1 and q
        return (float(u[q1 - 1:q1 + 1, q1 - 1:q1 + 1].mean()), float(u[q3 - 1:q3 + 1, q3 - 1:q3 + 1].mean()))
    return pb, u0, probe


def run(name):
    pb, u0, probe = setup(name)
    t0 = time.time()
    nsteps = int(round(T_END / pb.dt))
    U = np.asarray(u0, dtype=np.float64)
    s0 = [np.sign(v) for v in probe(U)]
    cross = [None, None]
    for k in range(1, nsteps + 1):
        U, _ = FP.ch_implicit_step(pb, U)
        vals = probe(U)
        for q in range(2):
            if cross[q] is None and np.sign(vals[q]) != s0[q]:
                cross[q] = k
        if all(c is not None for c in cross):
            break
    iv = [None if c is None else [round((c - 1) * pb.dt, 6), round(c * pb.dt, 6)] for c in cross]
    return name, {"a": pb.a, "b": pb.b, "dt": pb.dt, "n": pb.nx, "T1_interval": iv[0], "T2_interval": iv[1],
                  "cpu_seconds": round(time.time() - t0, 1)}


def main():
    names = sys.argv[1:] or list(READINGS)
    path = os.path.join(HERE, "seven_circles_readings.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    out["cite"] = ("Section 3.2.1 and Table 1 (seven circles); the paper prints T1 in [6.340, 6.345] and "
                   "T2 in [26.015, 26.020].  Each reading changes one thing against the baseline; crossing "
                   "times are intervals [(s - 1) h_t, s h_t] of the first step s after which u has changed "
                   "sign (null: no change by t = 30).  Solved by oracle/fixed_point.py.")
    readings = out.setdefault("readings", {})
    with mp.get_context("spawn").Pool(min(len(names), os.cpu_count() or 1)) as pool:
        for name, res in pool.imap_unordered(run, names):
            readings[name] = res
            print(name, res, flush=True)
            json.dump(out, open(path, "w"), indent=1)


if __name__ == "__main__":
    main()
