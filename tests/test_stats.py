"""Statistics of a tally and the figure of merit against hand-computed values
and textbook identities (no GPU)."""

import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import stats


def test_relvar_of_sum_hand_values():
    # constant weights: no variance
    assert stats.relvar_of_sum(4, 4.0, 4.0) == 0.0
    # weights (0, 2, 0, 2): m = 1, per-ray variance 1, variance of the mean 1/4
    assert stats.relvar_of_sum(4, 4.0, 8.0) == pytest.approx(0.25, rel=1e-15)
    # one hit of weight 1 in 10 rays: m = 0.1, (0.1 - 0.01)/10 / 0.01 = 0.9
    assert stats.relvar_of_sum(10, 1.0, 1.0) == pytest.approx(0.9, rel=1e-14)
    assert stats.relvar_of_sum(10, 0.0, 0.0) == math.inf
    with pytest.raises(ValueError):
        stats.relvar_of_sum(0, 1.0, 1.0)


def test_batch_means_hand_values():
    m, rv = stats.relvar_batch_means([1.0, 2.0, 3.0])
    assert m == 2.0 and rv == pytest.approx(1.0 / 4.0)         # s^2 = 1
    assert stats.relvar_of_batch_mean([1.0, 2.0, 3.0]) == pytest.approx(1.0 / 12.0)
    with pytest.raises(ValueError):
        stats.relvar_batch_means([1.0])


def test_the_two_relvar_estimates_agree_on_bernoulli_runs():
    """K = 32 runs of n Bernoulli(p) rays: the moment formula gives
    (1 - p)/(n p) exactly in expectation; batch means agree within their own
    sampling error (relative sd sqrt(2/(K-1)) ~ 0.25 at K = 32)."""
    rng = np.random.default_rng(3)
    n, p, K = 20_000, 0.3, 32
    hits = rng.binomial(n, p, size=K)
    est = hits / n
    theory = (1 - p) / (n * p)
    per_run = [stats.relvar_of_sum(n, float(h), float(h)) for h in hits]
    assert np.mean(per_run) == pytest.approx(theory, rel=0.02)
    _, rv = stats.relvar_batch_means(est)
    assert abs(rv / theory - 1.0) < 4 * math.sqrt(2.0 / (K - 1))


def test_per_bin_and_secondary():
    n = 100
    sw = np.array([10.0, 1.0, 1e-6, 0.0])
    sw2 = np.array([20.0, 1.0, 1e-12, 0.0])
    r = stats.per_bin_relvar(n, sw, sw2)
    # bins above 1e-3 x max: the first two
    assert r.size == 2
    assert r[0] == pytest.approx((0.2 - 0.01) / n / 0.01)
    assert r[1] == pytest.approx((0.01 - 1e-4) / n / 1e-4)
    assert stats.secondary_relvar(n, sw, sw2) == pytest.approx(np.median(r))


def test_fom_and_amortisation():
    assert stats.fom(0.25, 2.0) == pytest.approx(2.0)
    # a 10 s set-up shared by 5 runs of 2 s: each charged 4 s
    assert stats.fom_amortised(0.25, 2.0, 10.0, 5) == pytest.approx(1.0)
    with pytest.raises(ValueError):
        stats.fom(0.0, 1.0)


def test_break_even_hand_values():
    # A: c_A = 1 (relvar 1e-6 at 1e6 rays), rate 1 ray/s, set-up 10 s;
    # B: c_B = 4, rate 2 rays/s: c_B/r_B - c_A/r_A = 1, so N = 10
    assert stats.break_even_rays(1e-6, 10**6, 1.0, 10.0, 4e-6, 10**6, 2.0) == pytest.approx(10.0)
    # at N rays the two FOMs are equal
    N = 10.0
    fa = 1.0 / ((1.0 / N) * (N / 1.0 + 10.0))
    fb = 1.0 / ((4.0 / N) * (N / 2.0))
    assert fa == pytest.approx(fb)
    # A slower per unit variance: never breaks even
    assert stats.break_even_rays(1e-6, 10**6, 1.0, 10.0, 1e-6, 10**6, 2.0) == math.inf


def test_z_score():
    assert stats.z_score(1.0, 0.01, 1.0, 0.01) == 0.0
    assert stats.z_score(1.1, 0.0025, 1.0, 0.0) == pytest.approx(0.1 / 0.055)
