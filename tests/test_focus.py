"""Pins of the oracle's focusing instrument (Sec. 3.2): the contract's
logarithm against the library one, the Gaussian source's deviates against
the normal law, and the compound refractive lens against Snell's law and
the focal length R / (2 N delta) of a thin-lens stack."""

import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

MM = 1e-3


def lens(n=16, delta0=wl.BE_DELTA_23, radius=200e-6, thickness=50e-6, aperture=0.5 * MM):
    return dict(radius=radius, thickness=thickness, aperture=aperture, n_lenses=n, delta0=delta0,
                e_ref=23.32, pitch=thickness + aperture * aperture / radius)


def test_ln_against_the_library(orc):
    rng = np.random.default_rng(1)
    x = np.exp(rng.uniform(-40, 40, 2000))
    for v in x:
        ref = math.log(v)
        assert abs(orc.ln64(v) - ref) <= 4e-16 * abs(ref) + 1e-18
        v32 = float(np.float32(v))
        assert abs(orc.ln32(v32) - math.log(v32)) <= 3e-7 * abs(math.log(v32)) + 2e-8
    for v in np.linspace(0.5, 2.0, 301):        # around 1, where ln x is small
        assert abs(orc.ln64(v) - math.log(v)) <= 1e-17 + 3e-16 * abs(math.log(v))
    assert orc.ln64(1.0) == 0.0 and orc.ln32(1.0) == 0.0
    assert orc.ln64(2.0) == 0.6931471805599453       # e = 1, m = 1: the constant itself


def test_gaussian_source_deviates(orc):
    """Spot positions and energies of the Gaussian source follow the normal
    law (KS test); the divergence weight is exp(-theta^2 / 2 sigma'^2)."""
    scipy = pytest.importorskip("scipy.stats")
    spec = wl.focusing_instrument()
    src = spec.components[0]
    st = orc.sample_starts(spec, 0, 20000, 5).astype(np.float64)
    assert scipy.kstest(st[0] / src["sigma_x"], "norm").pvalue > 1e-3
    assert scipy.kstest(st[1] / src["sigma_y"], "norm").pvalue > 1e-3
    assert scipy.kstest((st[2] - src["e0"]) / src["sigma_e"], "norm").pvalue > 1e-3
    D = src["target_dist"]
    ax = (st[3] - st[0]) / (D * src["div_x"])
    ay = (st[4] - st[1]) / (D * src["div_y"])
    np.testing.assert_allclose(st[5], np.exp(-0.5 * (ax * ax + ay * ay)), rtol=2e-6, atol=1e-30)




@pytest.mark.parametrize("mode", [64, 32])
def test_lens_on_axis_and_symmetry(orc, mode):
    L = lens()
    ok, x, k, path = orc.lens_ray(L, (0, 0, -0.1), (0, 0, 1), 23.32, mode)
    # the axis is kept exactly; in binary32 k_z moves by an ulp or so per
    # surface (1 + eta - 1 rounds), which no position depends on
    assert ok and k[0] == 0 and k[1] == 0 and x[0] == 0 and x[1] == 0
    assert k[2] == 1.0 if mode == 64 else abs(k[2] - 1.0) < 1e-6
    assert path == pytest.approx(16 * 50e-6, rel=1e-12 if mode == 64 else 1e-5)
    # mirror images: the exit of (-h, 0) is the exact mirror of (h, 0)
    a = orc.lens_ray(L, (1e-4, 0, -0.1), (0, 0, 1), 23.32, mode)
    b = orc.lens_ray(L, (-1e-4, 0, -0.1), (0, 0, 1), 23.32, mode)
    assert a[0] and b[0]
    assert a[2][0] == -b[2][0] and a[2][1] == 0.0 and b[2][1] == 0.0 and a[2][2] == b[2][2]
    assert a[1][0] == -b[1][0]


def test_single_lens_deflection_and_thickness(orc):
    """One double-sided lens deflects a parallel ray at height h by
    -2 delta h / R (paraxial), and the ray crosses the material thickness
    d + h^2 / R at that height."""
    for h in (20e-6, 100e-6, 300e-6):
        ok, x, k, path = orc.lens_ray(lens(n=1), (h, 0, -0.01), (0, 0, 1), 23.32, 64)
        assert ok
        assert k[0] == pytest.approx(-2 * wl.BE_DELTA_23 * h / 200e-6, rel=2e-3)
        assert path == pytest.approx(50e-6 + h * h / 200e-6, rel=1e-5)
        assert math.sqrt(k @ k) == pytest.approx(1.0, abs=1e-15)


def test_stack_focal_length_and_chromatic_scaling(orc):
    """Parallel rays cross the axis R / (2 N delta) behind the stack's centre
    (thick-lens and aberration corrections below 0.5 %), and the focal length
    scales as E^2 (delta ~ E^-2)."""
    def focus(E, h=50e-6):
        ok, x, k, _ = orc.lens_ray(lens(), (h, 0, -0.05), (0, 0, 1), E, 64)
        assert ok and k[0] < 0
        return x[2] + x[0] / -k[0] * k[2]
    f = 200e-6 / (2 * 16 * wl.BE_DELTA_23)
    assert focus(23.32) == pytest.approx(f, rel=5e-3)
    assert focus(26.0) / focus(20.0) == pytest.approx((26.0 / 20.0) ** 2, rel=5e-3)
    # outside the aperture the frame absorbs the ray
    assert not orc.lens_ray(lens(), (0.6 * MM, 0, -0.05), (0, 0, 1), 23.32, 64)[0]


def test_mode32_lens_follows_mode64(orc):
    rng = np.random.default_rng(3)
    for _ in range(50):
        x = (rng.uniform(-3e-4, 3e-4), rng.uniform(-3e-4, 3e-4), -0.02)
        k = np.array([rng.normal(0, 1e-5), rng.normal(0, 1e-5), 1.0])
        k /= np.linalg.norm(k)
        a = orc.lens_ray(lens(), x, k, 23.32, 64)
        b = orc.lens_ray(lens(), x, k, 23.32, 32)
        assert a[0] == b[0]
        if a[0]:
            # the stack's deflection (~1e-5 rad) survives binary32 to 1e-3
            np.testing.assert_allclose(b[2][:2] - k[:2], a[2][:2] - k[:2], rtol=2e-3, atol=2e-10)


def test_focusing_concentrates_the_beam(orc):
    """Through the 0.1 mm slit 14 m behind the lens pass far more rays with
    the lenses refracting than with delta = 0 (a plain aperture)."""
    n = 20000
    on = orc.trace(wl.focusing_instrument(), 0, n, 2, 64)
    off = orc.trace(wl.focusing_instrument(delta0=0.0), 0, n, 2, 64)
    n_on, n_off = on.monitor(3)[0].sum(), off.monitor(3)[0].sum()
    assert n_on > 0.5 * n and n_on > 20 * max(n_off, 1)
