"""Statistics of a Monte Carlo tally and the figure of merit (host, binary64).

A monitor bin holds N, sum p and sum p^2 over the rays traced (paper Sec.
2.2.2); the intensity estimate is I = sum p / N_emit (the mean weight per
emitted ray).  The precision of an estimate is its relative variance, and the
figure of merit FOM = 1 / (relative variance x seconds) compares methods that
spend time differently: it does not depend on the run length for an unbiased
estimator whose variance falls as 1/N.

Two estimates of the relative variance of one run's mean:
* from the run's own moments: var = (sum p^2 / n - m^2) / n, m = sum p / n;
* by batch means: K runs under independent seeds give K estimates x_k; their
  sample variance (n - 1 denominator) is the variance of one run's estimate.
The first needs one run, the second no assumption about the per-ray
distribution beyond independence of the runs; they must agree.
"""

from __future__ import annotations

import math

import numpy as np


def relvar_of_sum(n: int, sw: float, sw2: float) -> float:
    """Relative variance of the mean weight per ray over n rays from its
    first two moments (inf when the mean is not positive)."""
    if n <= 0:
        raise ValueError("n must be positive")
    m = sw / n
    var = max(sw2 / n - m * m, 0.0) / n
    return var / (m * m) if m > 0 else math.inf


def relvar_batch_means(estimates) -> tuple[float, float]:
    """(mean, relative variance of ONE run's estimate) from K >= 2 independent
    runs' estimates, by their sample variance."""
    x = np.asarray(estimates, dtype=np.float64)
    if x.size < 2:
        raise ValueError("batch means need at least two runs")
    m = float(x.mean())
    var = float(x.var(ddof=1))
    return m, (var / (m * m) if m > 0 else math.inf)


def relvar_of_batch_mean(estimates) -> float:
    """Relative variance of the mean of all K runs (one run's / K)."""
    x = np.asarray(estimates, dtype=np.float64)
    return relvar_batch_means(x)[1] / x.size


def per_bin_relvar(n: int, sw, sw2, floor: float = 1e-3) -> np.ndarray:
    """Relative variance of each bin's mean weight per ray over n rays, for
    the bins whose estimate exceeds `floor` x the largest bin's (the others
    are dropped)."""
    sw = np.asarray(sw, dtype=np.float64)
    sw2 = np.asarray(sw2, dtype=np.float64)
    m = sw / n
    keep = m > floor * m.max() if m.size and m.max() > 0 else np.zeros(m.shape, dtype=bool)
    mk = m[keep]
    var = np.maximum(sw2[keep] / n - mk * mk, 0.0) / n
    return var / (mk * mk)


def secondary_relvar(n: int, sw, sw2, floor: float = 1e-3) -> float:
    """Median per-bin relative variance over the bins above `floor` x max."""
    r = per_bin_relvar(n, sw, sw2, floor)
    return float(np.median(r)) if r.size else math.inf


def fom(relvar: float, seconds: float) -> float:
    """Figure of merit 1 / (relative variance x seconds)."""
    if relvar <= 0 or seconds <= 0:
        raise ValueError("relvar and seconds must be positive")
    return 1.0 / (relvar * seconds)


def fom_amortised(relvar: float, seconds: float, setup_seconds: float, runs: int) -> float:
    """FOM of one run when a one-off set-up (training a proposal) is shared
    by `runs` runs: each run is charged setup_seconds / runs."""
    return fom(relvar, seconds + setup_seconds / max(int(runs), 1))


def break_even_rays(relvar_a: float, rays_a: int, rate_a: float, setup_a: float,
                    relvar_b: float, rays_b: int, rate_b: float) -> float:
    """Rays method A must trace after a one-off set-up of setup_a seconds
    before its FOM, set-up included, equals method B's (no set-up).  With
    relvar = c / N, method X's FOM over N rays is 1 / (c_X / rate_X +
    c_X setup_X / N); equal FOMs give N = c_A setup_A / (c_B / rate_B -
    c_A / rate_A).  inf when A is not faster per unit variance even without
    its set-up."""
    ca = relvar_a * rays_a
    cb = relvar_b * rays_b
    gap = cb / rate_b - ca / rate_a
    if gap <= 0:
        return math.inf
    return ca * setup_a / gap


def z_score(mean_a: float, relvar_a: float, mean_b: float, relvar_b: float) -> float:
    """Difference of two independent estimates in units of its standard
    deviation (relvar of each estimate given)."""
    var = relvar_a * mean_a * mean_a + relvar_b * mean_b * mean_b
    return (mean_a - mean_b) / math.sqrt(var) if var > 0 else math.inf
