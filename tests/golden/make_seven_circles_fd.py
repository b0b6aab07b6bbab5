"""Write seven_circles_fd.json: the steps at which the implicit five-point-Laplacian scheme of
Section 3.2.1's seven-circle example (Table 1; a = 0.1^2, b = 1, N_x = 128, h_t = 1/200)
changes sign at (pi/2, pi/2) and (3pi/2, 3pi/2).  Calls only ``oracle/`` (the fixed-point
solver of oracle/fixed_point.py) and the seeded-input module; takes about ten minutes.

    python tests/golden/make_seven_circles_fd.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fixed_point as FP  # noqa: E402
from paper_2305_03945_gb300 import workloads as WL  # noqa: E402


def main():
    w = WL.config_seven_circles(128)
    t0 = time.time()
    s1, s2 = FP.sign_change_steps(w.problem, w.u0, [(32, 32), (96, 96)], 6000)
    out = {
        "cite": "Section 3.2.1 and Table 1 (seven circles), solved by the oracle's fixed-point implicit step "
                "(oracle/fixed_point.py) to max |dU| <= 1e-14 per step; the paper prints T1 in [6.340, 6.345] "
                "and T2 in [26.015, 26.020]",
        "dt": w.problem.dt, "n": 128,
        "T1_step": s1, "T2_step": s2,
        "T1_interval": [(s1 - 1) * w.problem.dt, s1 * w.problem.dt],
        "T2_interval": [(s2 - 1) * w.problem.dt, s2 * w.problem.dt],
        "cpu_seconds": round(time.time() - t0, 1),
    }
    json.dump(out, open(os.path.join(HERE, "seven_circles_fd.json"), "w"), indent=1)
    print(out)


if __name__ == "__main__":
    main()
