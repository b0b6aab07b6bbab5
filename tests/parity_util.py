"""Shared checks of the GPU parity tests.

The stopping rule of Section 2.1 stops at the first iterate U_n whose measure is <= the
threshold (ties go to "stop").  The CUDA path and the oracle evaluate that measure on iterates
that agree to rounding, so their iteration counts must be equal -- unless the measure of the
iterate at which one of them stops lies so close to the threshold that rounding decides the
comparison.  ``assert_same_iterations`` accepts a count that differs by one only in that case:
the GPU's and the oracle's measures of the SAME iterate (the earlier of the two stopping
iterates) lie on opposite sides of the threshold and differ from each other by at most
``TIE_BAND`` of it.  A PDHG update changes the measure by a whole contraction factor (typically
0.3-0.9), so an off-by-one in either stopping rule cannot pass as a tie.
"""
import numpy as np

from oracle import rd_oracle as O

TIE_BAND = 1e-3


def threshold(pb, uk):
    """The oracle's stopping threshold for U^k (delta, or tol ||U^k||_2)."""
    return O.measure(pb, np.zeros(pb.shape), np.asarray(uk, dtype=np.float64))[1]


def assert_same_iterations(n_gpu, info_ref, pb, uk, gpu_measure_at):
    """n_gpu: the GPU's iteration count; info_ref: the oracle's pdhg_step info with history;
    gpu_measure_at(m): the GPU's stopping measure of its iterate m (from a run capped at m
    updates, or the measure it returned when m is its own stopping iterate)."""
    n_ref = info_ref["iterations"]
    if n_gpu == n_ref:
        return
    assert abs(n_gpu - n_ref) == 1, ("iteration counts differ by more than a tie", n_gpu, n_ref)
    m = min(n_gpu, n_ref)
    thr = threshold(pb, uk)
    r_ref = float(info_ref["history"][m])
    r_gpu = float(gpu_measure_at(m))
    assert (r_gpu - thr) * (r_ref - thr) <= 0.0, ("not a tie: both measures on one side", r_gpu, r_ref, thr)
    assert abs(r_gpu - r_ref) <= TIE_BAND * thr, ("not a tie: measures of one iterate differ", r_gpu, r_ref, thr)
