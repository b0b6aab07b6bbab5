"""The seeded synthetic inputs (paper_2305_03945_gb300/workloads.py), CPU only: the serving mix
follows its stated recipe, is reproducible, and adding the 3-D requests leaves every square-grid
request unchanged.  Grids are shrunk here (the draws do not depend on the side values), so the
4000-request mix is checked without allocating it."""
import numpy as np

from paper_2305_03945_gb300 import workloads as WL

TINY = (4, 8, 4, 8, 4)          # five sides, as in the mix: the same random draws, small arrays


def test_full_mix_recipe():
    reqs = WL.serving_requests(4000, sides=TINY, cube=4)
    cubes = [pb for pb, _, _ in reqs if pb.nz > 1]
    assert len(reqs) == 4000 and len(cubes) == 698        # the count the serving notes quote
    kinds = [pb.kind for pb, _, _ in reqs]
    assert set(kinds) == {"allen_cahn", "ch_split"}
    assert abs(kinds.count("allen_cahn") / 4000 - 0.5) < 0.03
    bcs = [pb.bc for pb, _, _ in reqs]
    assert abs(bcs.count("periodic") / 4000 - 0.5) < 0.03
    steps = [n for _, _, n in reqs]
    assert min(steps) == 10 and max(steps) == 50
    assert all(pb.tol == 1e-6 and pb.tol_kind == "f_rel" for pb, _, _ in reqs)
    for pb, u0, _ in reqs[:200]:
        assert u0.shape == pb.shape
        if pb.kind == "ch_split":
            # U[-0.1, 0.1] minus its mean
            assert abs(u0.mean()) < 1e-12 and np.max(u0) - np.min(u0) <= 0.2
        else:
            assert np.max(np.abs(u0)) <= 0.05


def test_mix_is_reproducible_and_cubes_leave_square_requests_unchanged():
    a = WL.serving_requests(300, sides=TINY, cube=4)
    b = WL.serving_requests(300, sides=TINY, cube=4)
    flat = WL.serving_requests(300, sides=TINY, cube=None)
    for (pa, ua, na), (pb_, ub, nb), (pf, uf, nf) in zip(a, b, flat):
        assert pa == pb_ and na == nb and np.array_equal(ua, ub)
        if pa.nz == 1:
            assert pa == pf and na == nf and np.array_equal(ua, uf)
        else:
            assert (pa.nx, pa.ny, pa.nz) == (4, 4, 4) and pf.nz == 1


def test_poisson_arrivals_have_the_rate():
    t = WL.poisson_arrivals(20000, rate=8.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() * 8.0 - 1) < 0.03
    assert np.array_equal(t, WL.poisson_arrivals(20000, rate=8.0))


def test_gray_scott_patches_recipe():
    """u = 1, v = 0 outside the patches, (0.5, 0.25) inside, each value within 1% noise; the
    patches (side n / 12.8, 10 of them, possibly overlapping) cover at most 10 side^2 points."""
    n = 128
    U = WL.gray_scott_patches(4000, n)
    u, v = U[0], U[1]
    assert U.shape == (2, n, n)
    inside = v > 0
    assert np.all(np.abs(u[~inside] - 1) <= 0.01 + 1e-15) and np.all(v[~inside] == 0)
    assert np.all(np.abs(u[inside] / 0.5 - 1) <= 0.01 + 1e-15) and np.all(np.abs(v[inside] / 0.25 - 1) <= 0.01 + 1e-15)
    side = round(n / 12.8)
    assert side * side <= inside.sum() <= 10 * side * side


def test_smoothed_tanh_recipe():
    """tanh of smoothed noise scaled by its standard deviation: values in (-1, 1), zero-mean to
    sampling error, and smooth on the 8-cell scale (neighbour differences far below the range)."""
    u = WL.smoothed_tanh(2000, 256, 256)
    assert u.shape == (256, 256) and np.all(np.abs(u) < 1)
    assert abs(u.mean()) < 0.2
    assert np.max(np.abs(np.diff(u, axis=1))) < 0.25 * (u.max() - u.min())
    assert np.array_equal(u, WL.smoothed_tanh(2000, 256, 256))
