"""Pins of the oracle's scattering phantom (Sec. 3.3: each step of the
fixed-step march updates the weight and may change the direction): the
event sampler against the Rayleigh (Thomson) and Klein-Nishina laws and the
Compton energy shift, the process choice, the unscattered
fraction of a pencil beam against exp(-mu_s L), weight conservation without
absorption, and the zero-coefficient limit against the plain march."""

import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

MM = 1e-3


def _samples(orc, n, mr, mc, k, E, mode):
    out = [orc.scatter_dir(i, 3, 11, 0, mr, mc, k, E, mode) for i in range(n)]
    return np.array([o[0] for o in out]), np.array([o[1] for o in out])


@pytest.mark.parametrize("mode", [64, 32])
def test_rayleigh_polar_law(orc, mode):
    """Elastic events: cos(theta) follows (3/8)(1 + mu^2) (KS), the energy
    is kept, the azimuth is uniform, |k'| = 1."""
    scipy = pytest.importorskip("scipy.stats")
    ks, Es = _samples(orc, 20000, 20.0, 0.0, (0.0, 0.0, 1.0), 60.0, mode)
    mu = ks[:, 2]
    cdf = lambda m: 0.5 + 0.375 * (m + m ** 3 / 3.0)
    assert scipy.kstest(mu, cdf).pvalue > 1e-3
    assert (Es == 60.0).all()
    phi = (np.arctan2(ks[:, 1], ks[:, 0]) + math.pi) / (2 * math.pi)
    assert scipy.kstest(phi, "uniform").pvalue > 1e-3
    tol = 1e-15 if mode == 64 else 3e-7
    assert np.abs(np.linalg.norm(ks, axis=1) - 1.0).max() < 8 * tol


@pytest.mark.parametrize("mode", [64, 32])
def test_compton_klein_nishina(orc, mode):
    """Compton events at 100 keV on a tilted ray: the angle to the old
    direction follows Klein-Nishina (KS against the law integrated
    numerically) and the energy is E / (1 + (E/m_e c^2)(1 - cos theta))."""
    scipy = pytest.importorskip("scipy.stats")
    E = 100.0
    k0 = np.array([0.3, -0.2, 0.9])
    k0 /= np.linalg.norm(k0)
    ks, Es = _samples(orc, 20000, 0.0, 30.0, k0, E, mode)
    mu = ks @ k0
    kk = E / 510.99895
    g = np.linspace(-1, 1, 200001)
    e = 1.0 / (1.0 + kk * (1.0 - g))
    pdf = e * e * (e + 1.0 / e - (1.0 - g * g))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (pdf[1:] + pdf[:-1]) * np.diff(g))])
    cdf /= cdf[-1]
    assert scipy.kstest(np.clip(mu, -1, 1), lambda m: np.interp(m, g, cdf)).pvalue > 1e-3
    rel = 1e-12 if mode == 64 else 2e-6
    np.testing.assert_allclose(Es, E / (1.0 + kk * (1.0 - mu)), rtol=rel)
    assert (Es < E).mean() > 0.99


def test_process_choice(orc):
    """The event is Compton with probability mu_C / (mu_R + mu_C)."""
    n = 20000
    _, Es = _samples(orc, n, 10.0, 30.0, (0.0, 0.0, 1.0), 80.0, 64)
    frac = (Es < 80.0).mean()      # Compton lowers E (a forward Compton event keeps it: rare)
    assert abs(frac - 0.75) < 5 * math.sqrt(0.75 * 0.25 / n) + 2e-3


def pencil_block(mu_s, absorb=False, uniform=True, **kw):
    spec = wl.scatter_block(mu_s=mu_s, absorb=absorb, det_n=200, **kw)
    spec.components[0]["target_w"] = 0.0
    spec.components[0]["target_h"] = 0.0
    if uniform:
        spec.phantom[:] = 1
    return spec


@pytest.mark.parametrize("mode,compton", [(64, 0.0), (32, 0.0), (64, 2.0)])
def test_unscattered_fraction(orc, mode, compton):
    """A pencil along the axis of a uniform block: it stays unscattered with
    probability exp(-(mu_R + mu_C) L) (the march's step lengths add up to L),
    and only unscattered rays reach the detector's central bin."""
    mu_s, L, n = 20.0, 20 * 2 * MM, 20000
    r = orc.trace(pencil_block(mu_s, compton=compton), 0, n, 5, mode)
    N = r.monitor(2)[0].reshape(200, 200)
    p = math.exp(-mu_s * (1.0 + compton) * L)
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


@pytest.mark.parametrize("E", [1.0, 40.0, 150.0])
def test_klein_nishina_total_matches_the_integrated_law(E):
    """The synthetic Compton tables' cross-section: the closed form equals
    the Klein-Nishina differential law, r_e^2/2 e^2 (e + 1/e - sin^2),
    integrated over the sphere, and tends to the Thomson 8 pi r_e^2 / 3 as
    E -> 0."""
    g = np.linspace(-1.0, 1.0, 400001)
    e = 1.0 / (1.0 + E / wl.ME_C2 * (1.0 - g))
    d = 0.5 * wl.R_E ** 2 * e * e * (e + 1.0 / e - (1.0 - g * g))
    integral = 2.0 * math.pi * float(np.sum(0.5 * (d[1:] + d[:-1]) * np.diff(g)))
    assert wl.klein_nishina_sigma(E) == pytest.approx(integral, rel=1e-9)
    thomson = 8.0 * math.pi / 3.0 * wl.R_E ** 2
    k = 0.01 / wl.ME_C2
    assert wl.klein_nishina_sigma(0.01) == pytest.approx(thomson * (1.0 - 2.0 * k), rel=1e-6)


def test_tabulated_curves_pass_through_the_cell_ends():
    """Each cell's line of the water tables meets its curve at both ends."""
    ray, com = wl.water_scattering(e_min=20.0, e_max=120.0, n_cell=50)
    e = 20.0 + 2.0 * np.arange(51)
    for t, f in ((ray[1], lambda x: 1.2 * (40.0 / x) ** 2),
                 (com[2], lambda x: 2.0 * wl.WATER_NE * wl.klein_nishina_sigma(x))):
        np.testing.assert_allclose(t[:, 0] + t[:, 1] * e[:-1], f(e[:-1]), rtol=1e-12)
        np.testing.assert_allclose(t[:, 0] + t[:, 1] * e[1:], f(e[1:]), rtol=1e-12)


@pytest.mark.parametrize("mode", [64, 32])
@pytest.mark.parametrize("E", [30.0, 90.0])
def test_energy_dependent_unscattered_fraction(orc, mode, E):
    """Energy-dependent tables (Rayleigh ~ E^-2, Compton ~ Klein-Nishina): a
    nearly monochromatic pencil at E stays unscattered with probability
    exp(-(mu_R(E) + mu_C(E)) L), the coefficients taken at the ray's energy
    (at 30 keV 2.6 times the depth at 90 keV)."""
    mu_s, L, n = 20.0, 20 * 2 * MM, 20000
    spec = pencil_block(mu_s, compton=1.0, energy_dependent=True)
    spec.components[0]["e_min"], spec.components[0]["e_max"] = E - 0.01, E + 0.01
    r = orc.trace(spec, 0, n, 5, mode)
    N = r.monitor(2)[0].reshape(200, 200)
    mu = mu_s * (40.0 / E) ** 2 + mu_s * wl.klein_nishina_sigma(E) / wl.klein_nishina_sigma(40.0)
    p = math.exp(-mu * L)
    assert abs(N[100, 100] / n - p) < 5 * math.sqrt(p * (1 - p) / n) + 1e-3


def test_zero_slope_tables_equal_constant_coefficients(orc):
    """Coefficients given per material and the same values as zero-slope
    per-cell tables trace identically (the constant case of the tables)."""
    a = wl.scatter_block(mu_s=40.0, compton=1.5)
    b = wl.scatter_block(mu_s=40.0, compton=1.5)
    nc = b.materials.n_cell
    b.mu_scatter = np.stack([np.repeat(a.mu_scatter[:, None], nc, 1), np.zeros((3, nc))], -1)
    b.mu_compton = np.stack([np.repeat(a.mu_compton[:, None], nc, 1), np.zeros((3, nc))], -1)
    for mode in (64, 32):
        ra, rb = orc.trace(a, 0, 4000, 3, mode), orc.trace(b, 0, 4000, 3, mode)
        for i in range(3):
            assert np.array_equal(ra.monitor(2)[i], rb.monitor(2)[i])


def compton_step_block():
    """A uniform block scattering by Compton only, 50 /m at E >= 95 keV and
    1 /m below (a step on a cell boundary), lit by a 100 keV pencil; an
    energy monitor of 1000 bins over 20-120 keV, 2 x 2 m, behind it."""
    s = wl.scatter_block(mu_s=0.0, absorb=False)
    s.phantom[:] = 1
    src = s.components[0]
    src["e_min"], src["e_max"] = 99.99, 100.01
    src["target_w"] = src["target_h"] = 0.0
    m = s.materials
    e_lo = m.e_min + (m.e_max - m.e_min) / m.n_cell * np.arange(m.n_cell)
    t = np.zeros((3, m.n_cell, 2))
    t[1, :, 0] = np.where(e_lo < 95.0 - 1e-9, 1.0, 50.0)
    s.mu_compton = t
    s.components[2] = wl.component("mon_e", pos=s.components[2]["pos"], ne=1000, e_min=20.0,
                                   e_max=120.0, xmin=-1.0, xmax=1.0, ymin=-1.0, ymax=1.0)
    return s


@pytest.mark.parametrize("mode", [64, 32])
def test_compton_energy_looks_up_the_scattering_ahead(orc, mode):
    """After a Compton event the scattering coefficients are taken at the
    new energy.  Compton only, 50 /m at E >= 95 keV and 1 /m below (a step
    on a cell boundary), on a 100 keV pencil: a ray that has fallen below
    95 keV scatters again with probability at most 1 - exp(-1 /m x 69 mm)
    < 7 % (69 mm: the block's diagonal), and only such a second event below
    95 keV can take it under 95 / (1 + 2 x 95 / m_e c^2) = 69.26 keV.  So
    under that floor lie at most 7 % of the rays detected below 95 keV; a
    march that kept the entry energy's 50 /m puts ~40 % there."""
    N = orc.trace(compton_step_block(), 0, 20000, 3, mode, threads=8).monitor(2)[0]
    e = 20.0 + 0.1 * np.arange(1000)
    floor = 95.0 / (1.0 + 2.0 * 95.0 / wl.ME_C2)
    below = N[e + 0.1 <= floor].sum()
    between = N[(e >= floor) & (e < 95.0)].sum()
    assert between > 1000
    assert below <= 0.07 * (below + between)
