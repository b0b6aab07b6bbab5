"""The iteration-count rule the GPU parity tests apply (tests/parity_util.py), CPU only: equal
counts pass; a count one apart passes only when the two measures of the same iterate straddle
the threshold within the tie band; anything else fails."""
import numpy as np
import pytest

from paper_2305_03945_gb300 import workloads as WL
from parity_util import TIE_BAND, assert_same_iterations

PB = WL.Problem(nx=4, ny=4, lx=1.0, ly=1.0, bc="periodic", op="laplacian", kind="none", dt=1.0,
                tol=1.0, tol_kind="res_abs")   # threshold delta = 1
UK = np.zeros(PB.shape)


def _ref(history):
    return {"iterations": len(history) - 1, "history": np.array(history, dtype=float)}


def test_equal_counts_pass():
    assert_same_iterations(3, _ref([9.0, 4.0, 2.0, 0.5]), PB, UK, lambda m: 99.0)


@pytest.mark.parametrize("n_gpu", [1, 5])
def test_counts_two_apart_fail(n_gpu):
    with pytest.raises(AssertionError, match="more than a tie"):
        assert_same_iterations(n_gpu, _ref([9.0, 4.0, 2.0, 0.5]), PB, UK, lambda m: 1.0)


def test_a_tie_passes_either_way():
    # the oracle stops at 3 (its measure of iterate 2 is just above delta); the GPU's measure of
    # the same iterate 2 is just below: the GPU stops at 2
    ref = _ref([9.0, 4.0, 1.0 + 0.2 * TIE_BAND, 0.5])
    assert_same_iterations(2, ref, PB, UK, lambda m: 1.0 - 0.2 * TIE_BAND)
    # the oracle stops at 2 (its measure just below), the GPU at 3 (its measure of 2 just above)
    ref = _ref([9.0, 4.0, 1.0 - 0.2 * TIE_BAND])
    assert_same_iterations(3, ref, PB, UK, lambda m: 1.0 + 0.2 * TIE_BAND)


def test_both_measures_on_one_side_fail():
    ref = _ref([9.0, 4.0, 1.0 + 0.2 * TIE_BAND, 0.5])
    with pytest.raises(AssertionError, match="one side"):
        assert_same_iterations(2, ref, PB, UK, lambda m: 1.0 + 0.1 * TIE_BAND)


def test_an_off_by_one_of_a_whole_update_fails():
    # one contraction step apart (0.6): the measures straddle delta but far outside the band
    ref = _ref([9.0, 4.0, 1.3, 0.78])
    with pytest.raises(AssertionError, match="differ"):
        assert_same_iterations(2, ref, PB, UK, lambda m: 0.78)
