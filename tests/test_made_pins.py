"""Pins of the oracle's minimum theoretical MADE (supplementary material, the
section on the components found for different theta_c): closed forms worked by
hand, brute force over every breakpoint of the piecewise-linear error, the
textbook median for offsets, invariance to per-component scales and the
monotonicity of the minimum under coarsening of the partition."""
import itertools

import numpy as np
import pytest

import oracle as O


def test_closed_form_two_pixels():
    # perspective: r = g / d = (2, 1) with weights d = (1, 3); the weighted
    # median is 1 (weight 3 of 4), E = |1 - 2| + |3 - 3| = 1 over 2 pixels
    made, per, s = O.min_made(np.array([[1.0, 3.0]]), np.array([[2.0, 3.0]]), None, 1, O.PERSP)
    assert made == 0.5 and per[0] == 0.5 and s[0] == 1.0
    # equal weights: every s in [1, 3] gives E = 2
    made, _, s = O.min_made(np.array([[1.0, 1.0]]), np.array([[1.0, 3.0]]), None, 1, O.PERSP)
    assert made == 1.0 and 1.0 <= s[0] <= 3.0


def test_closed_form_weighted_by_pixel_counts():
    # component 0: three pixels, offsets r = g - d = (0, 1, 5) -> median 1, E = 1 + 0 + 4 = 5
    # component 1: one pixel -> E = 0; MADE = 5 / 4 (pixels), not the mean of per-component MADEs
    d = np.array([[0.0, 0.0, 0.0, 7.0]])
    g = np.array([[0.0, 1.0, 5.0, 2.0]])
    lab = np.array([[0, 0, 0, 1]])
    made, per, s = O.min_made(d, g, lab, 2, O.ORTHO)
    assert made == 1.25
    assert np.allclose(per, [5.0 / 3.0, 0.0])
    assert s[0] == 1.0 and s[1] == -5.0


def test_excluded_pixels_do_not_count():
    d = np.array([[1.0, np.nan, 2.0, 4.0, -1.0]])
    g = np.array([[1.0, 5.0, np.inf, 4.0, 3.0]])
    lab = np.array([[0, 0, 0, -1, 0]])
    made, per, _ = O.min_made(d, g, lab, 1, O.PERSP)   # only pixel 0 counts
    assert made == 0.0 and per[0] == 0.0
    made, _, _ = O.min_made(np.full((2, 2), np.nan), np.ones((2, 2)), None, 1, O.PERSP)
    assert np.isnan(made)
    _, per, s = O.min_made(np.ones((1, 2)), np.ones((1, 2)), np.array([[0, 0]]), 3, O.ORTHO)
    assert per[1] == 0.0 and np.isnan(s[1]) and np.isnan(s[2])


@pytest.mark.parametrize("camera", [O.PERSP, O.ORTHO])
def test_brute_force_over_breakpoints(camera):
    """The minimum of a convex piecewise-linear function lies at one of its
    breakpoints: evaluate the error at every breakpoint and on a dense grid."""
    rng = np.random.default_rng(7)
    for trial in range(40):
        n = int(rng.integers(1, 8))
        d = rng.uniform(0.2, 5.0, n)
        g = rng.uniform(0.2, 5.0, n)
        if trial % 3 == 0:
            d[: n // 2] = d[0]   # repeated values: ties among the breakpoints
            g[: n // 2] = g[0]
        made, per, s = O.min_made(d[None], g[None], None, 1, camera)
        f = (lambda t: np.abs(t * d - g).sum()) if camera == O.PERSP else (lambda t: np.abs(d + t - g).sum())
        r = g / d if camera == O.PERSP else g - d
        best = min(f(t) for t in r)
        assert abs(per[0] * n - best) <= 1e-12 * max(best, 1.0)
        assert abs(f(s[0]) - best) <= 1e-12 * max(best, 1.0)
        grid = np.linspace(r.min() - 1.0, r.max() + 1.0, 2001)
        assert min(f(t) for t in grid) >= best - 1e-12 * max(best, 1.0)
        assert made == pytest.approx(best / n, rel=1e-12, abs=1e-15)


def test_offsets_reduce_to_the_median():
    rng = np.random.default_rng(3)
    for n in (1, 3, 5, 9, 101):
        d = rng.normal(size=n)
        g = rng.normal(size=n)
        made, _, s = O.min_made(d[None], g[None], None, 1, O.ORTHO)
        r = g - d
        assert s[0] == np.median(r)   # odd n: the median is a data value
        assert made == pytest.approx(np.abs(r - np.median(r)).mean(), rel=1e-12)


@pytest.mark.parametrize("camera", [O.PERSP, O.ORTHO])
def test_exact_up_to_component_scales_is_zero(camera):
    rng = np.random.default_rng(11)
    H, W, K = 24, 20, 6
    lab = rng.integers(0, K, (H, W))
    g = rng.uniform(1.0, 3.0, (H, W))
    if camera == O.PERSP:
        d = g * rng.uniform(0.1, 10.0, K)[lab]
    else:
        d = g + rng.normal(size=K)[lab] * 5.0
    made, per, s = O.min_made(d, g, lab, K, camera)
    assert made < 1e-14 and np.all(per < 1e-14)


@pytest.mark.parametrize("camera", [O.PERSP, O.ORTHO])
def test_invariant_to_component_scales(camera):
    rng = np.random.default_rng(5)
    H, W, K = 30, 30, 9
    lab = rng.integers(0, K, (H, W))
    g = rng.uniform(1.0, 3.0, (H, W))
    d = g * rng.uniform(0.9, 1.1, (H, W)) if camera == O.PERSP else g + rng.normal(scale=0.1, size=(H, W))
    made0, per0, _ = O.min_made(d, g, lab, K, camera)
    d2 = d * rng.uniform(0.2, 5.0, K)[lab] if camera == O.PERSP else d + rng.normal(size=K)[lab]
    made1, per1, _ = O.min_made(d2, g, lab, K, camera)
    assert made1 == pytest.approx(made0, rel=1e-12)
    assert np.allclose(per1, per0, rtol=1e-12, atol=0)


@pytest.mark.parametrize("camera", [O.PERSP, O.ORTHO])
def test_coarsening_never_lowers_the_minimum(camera):
    """Merging components leaves fewer free scales: the minimum can only grow;
    one component for all pixels gives the MADE after the best global scale."""
    rng = np.random.default_rng(9)
    H, W, K = 32, 32, 12
    lab = rng.integers(0, K, (H, W))
    g = rng.uniform(1.0, 3.0, (H, W))
    d = g * rng.uniform(0.5, 2.0, K)[lab] * rng.uniform(0.95, 1.05, (H, W))
    if camera == O.ORTHO:
        d = g + rng.normal(size=K)[lab] + rng.normal(scale=0.05, size=(H, W))
    fine, _, _ = O.min_made(d, g, lab, K, camera)
    for pairs in itertools.islice(itertools.combinations(range(K), 2), 0, 66, 7):
        merged = np.where(lab == pairs[1], pairs[0], lab)
        coarse, _, _ = O.min_made(d, g, merged, K, camera)
        assert coarse >= fine - 1e-12
    glob, _, _ = O.min_made(d, g, None, 1, camera)
    assert glob >= fine - 1e-12
