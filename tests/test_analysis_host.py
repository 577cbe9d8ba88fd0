"""Host-side analysis behind the DT-SQA experiment (no GPU): the Gaussian
extreme-value median of the best of R runs (Eq. EVTmedianFinal), pinned by
the order-statistic identity and by sampling."""
import numpy as np
import pytest

from paper_2503_10302_gb300.ttt import evt_median_gaussian


@pytest.mark.parametrize("r", [1, 2, 4, 16, 64, 256])
def test_evt_median_equals_order_statistic_quantile(r):
    """The minimum of r draws has median mu + sd Phi^-1(1 - 2^(-1/r)),
    computed here through the normal quantile instead of erfc^-1."""
    stats = pytest.importorskip("scipy.stats")
    mu, sd = 0.013, 0.004
    want = mu + sd * stats.norm.ppf(1.0 - 0.5 ** (1.0 / r))
    assert evt_median_gaussian(mu, sd, r) == pytest.approx(want, rel=1e-12, abs=1e-15)


def test_evt_median_single_run_is_the_mean():
    assert evt_median_gaussian(0.7, 0.2, 1) == pytest.approx(0.7, abs=1e-15)


def test_evt_median_matches_sampled_minima():
    """10^5 groups of r = 16 draws: the sample median of the group minima
    lies within a few standard errors of the formula."""
    rng = np.random.default_rng(5)
    mu, sd, r = 1.0, 0.5, 16
    mins = rng.normal(mu, sd, size=(100_000, r)).min(axis=1)
    got = float(np.median(mins))
    # standard error of a sample median: 1 / (2 f(m) sqrt(n)), f from a
    # density estimate of the minima at their median
    h = 0.02
    f = float(np.mean(np.abs(mins - got) < h)) / (2 * h)
    se = 1.0 / (2 * f * np.sqrt(mins.size))
    assert abs(got - evt_median_gaussian(mu, sd, r)) < 5 * se


def test_evt_median_decreases_with_r():
    vals = [evt_median_gaussian(0.0, 1.0, r) for r in (1, 2, 4, 8, 16, 32)]
    assert all(b < a for a, b in zip(vals, vals[1:]))
