"""Pins of the oracle's scattering phantom (Sec. 3.3: each step of the
fixed-step march updates the weight and may change the direction): the
isotropic sampler against the uniform law on the sphere, the unscattered
fraction of a pencil beam against exp(-mu_s L), weight conservation without
absorption, and the zero-coefficient limit against the plain march."""

import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

MM = 1e-3


@pytest.mark.parametrize("mode", [64, 32])
def test_isotropic_directions(orc, mode):
    scipy = pytest.importorskip("scipy.stats")
    ks = np.array([orc.iso_dir(i, 3, 11, 0, mode)[0] for i in range(20000)])
    tol = 1e-15 if mode == 64 else 3e-7
    assert np.abs(np.linalg.norm(ks, axis=1) - 1.0).max() < 4 * tol
    assert scipy.kstest((ks[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    phi = (np.arctan2(ks[:, 1], ks[:, 0]) + math.pi) / (2 * math.pi)
    assert scipy.kstest(phi, "uniform").pvalue > 1e-3


def pencil_block(mu_s, absorb=False, uniform=True, **kw):
    spec = wl.scatter_block(mu_s=mu_s, absorb=absorb, det_n=200, **kw)
    spec.components[0]["target_w"] = 0.0
    spec.components[0]["target_h"] = 0.0
    if uniform:
        spec.phantom[:] = 1
    return spec


@pytest.mark.parametrize("mode", [64, 32])
def test_unscattered_fraction(orc, mode):
    """A pencil along the axis of a uniform block: it stays unscattered with
    probability exp(-mu_s L) (the march's step lengths add up to L), and only
    unscattered rays reach the detector's central bin."""
    mu_s, L, n = 20.0, 20 * 2 * MM, 20000
    r = orc.trace(pencil_block(mu_s), 0, n, 5, mode)
    N = r.monitor(2)[0].reshape(200, 200)
    p = math.exp(-mu_s * L)
    direct = N[100, 100]      # the axis hits the corner of four bins: (100, 100) on the half-open grid
    assert abs(direct / n - p) < 5 * math.sqrt(p * (1 - p) / n)
    assert N.sum() > direct   # scattered rays also reach the detector


def test_weight_conserved_without_absorption(orc):
    n = 10000
    r = orc.trace(wl.scatter_block(mu_s=50.0, absorb=False), 0, n, 7, 64)
    assert r.lost[1] == 0.0 and r.sum_w0 == n
    # every ray's weight ends alive or lost where it could not reach the
    # detector plane (scattered backwards)
    assert r.sum_wend + r.lost.sum() == pytest.approx(n, rel=1e-12)
    assert r.lost[2] > 0


@pytest.mark.parametrize("mode", [64, 32])
def test_zero_coefficients_equal_the_march(orc, mode):
    """mu_s = 0 everywhere: the scattering march is the plain march (same
    monitors bit for bit, the extra depth draw aside)."""
    a = wl.scatter_block(mu_s=0.0)
    b = wl.scatter_block(mu_s=0.0)
    b.components[1]["scatter"] = False
    ra, rb = orc.trace(a, 0, 5000, 3, mode), orc.trace(b, 0, 5000, 3, mode)
    assert np.array_equal(ra.monitor(2)[0], rb.monitor(2)[0])
    assert np.array_equal(ra.monitor(2)[1], rb.monitor(2)[1])


def test_many_scatterings_stop_after_eight(orc):
    """A dense scatterer (mean free path 0.1 mm in a 40 mm block): every ray
    scatters its eight times, none keeps its line, and all finish."""
    r = orc.trace(pencil_block(1e4), 0, 2000, 9, 64)
    N = r.monitor(2)[0].reshape(200, 200)
    assert N[100, 100] <= 2 and r.n_emit == 2000
