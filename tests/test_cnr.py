"""The CNR study of the paper's staircase test piece (Sec. 5.1) on the host:
the analysis against hand-computed values, the test piece's geometry against
its definition, and the oracle's transmission through one step against the
closed form w0 exp(-mu(E) t / k_z) of a slab."""

import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import cnr
from paper_2410_08747_gb300 import workloads as wl

MM = 1e-3


def test_cnr_closed_form():
    # region A: 1, 2, 3, 4 -> mean 2.5, s^2 = 5/3, s_mean^2 = 5/12
    # region B: 5, 5, 7, 7 -> mean 6,   s^2 = 4/3, s_mean^2 = 1/3
    # CNR = 3.5 / sqrt(5/12 + 4/12) = 3.5 / sqrt(0.75)
    a = np.array([1.0, 2.0, 3.0, 4.0]).reshape(2, 2, 1)
    b = np.array([5.0, 5.0, 7.0, 7.0]).reshape(2, 2, 1)
    assert cnr.cnr(a, b)[0] == pytest.approx(3.5 / math.sqrt(0.75), rel=1e-14)
    assert cnr.cnr(b, a)[0] == pytest.approx(3.5 / math.sqrt(0.75), rel=1e-14)


def test_normalisation_and_empty_flat_field():
    sw = np.array([[[2.0, 3.0]], [[4.0, 0.0]]])        # 2 lines, 1 pixel, 2 bins
    flat = np.array([[4.0, 0.0]])
    i = cnr.normalised(sw, flat)
    assert i[0, 0, 0] == 0.5 and i[1, 0, 0] == 1.0
    assert np.isnan(i[:, 0, 1]).all()


def test_fit_and_criterion():
    e = cnr.bin_centres(20.0, 160.0, 128)
    y = 0.5 + 0.02 * e
    a, b = cnr.fit_above(e, y, 80.0)
    assert a == pytest.approx(0.5, abs=1e-12) and b == pytest.approx(0.02, abs=1e-14)
    # three points, closed-form least squares: (80, 1), (100, 3), (120, 2)
    a, b = cnr.fit_above(np.array([60.0, 80.0, 100.0, 120.0]), np.array([9.0, 1.0, 3.0, 2.0]), 80.0)
    assert b == pytest.approx(1.0 / 40.0, rel=1e-12) and a == pytest.approx(2.0 - 100.0 / 40.0, rel=1e-12)
    assert cnr.passes(1.5, 0.001, 20.0, 160.0)
    assert not cnr.passes(0.5, 0.01, 20.0, 160.0)      # below 1 at 20 keV
    assert not cnr.passes(3.0, -0.015, 20.0, 160.0)    # below 1 at 160 keV


def test_staircase_geometry():
    v = 1 * MM
    ph = wl.staircase_phantom(v)
    nz, ny, nx = ph.shape
    sw = int(round(wl.STAIR_STEP_W / v))
    for k in range(wl.STAIR_N):
        t = int(round((wl.STAIR_T0 + k * wl.STAIR_DT) / v))
        col = ph[:, k * sw + sw // 2, 5]                 # a column away from the rod
        assert (col[:t] == 1).all() and (col[t:] == 0).all()
    # the rod: a disc of radius 5 voxels, the same in every y slice, below the steps
    disc = ph[:, 0, :] == 2
    assert (ph == 2).sum() == disc.sum() * ny
    zz, xx = np.nonzero(disc)
    assert zz.min() > round((wl.STAIR_T0 + (wl.STAIR_N - 1) * wl.STAIR_DT) / v)
    assert abs(disc.sum() - math.pi * 25) < 0.05 * math.pi * 25
    assert (xx + 0.5).mean() == pytest.approx(0.5 * nx)
    # step 6 (26 mm) is centred on the central detector's axis
    assert wl.staircase_step_y(6, v) == pytest.approx((6.5 * 20 - 100) * MM)


def test_oracle_transmission_through_one_step(orc):
    """Rays of a steel-only line that cross step 6 (26 mm of iron) inside its
    band: detected weight = w0 exp(-mu_iron(E) 0.026 / k_z)."""
    x_line = 10.5 * MM
    spec = wl.staircase_line(x_line, n_det=1, det_px=32, ne=16)
    n = 4000
    st = orc.sample_starts(spec, 0, n, 21)
    _, det = orc.trace_starts(spec, st)
    src, ph = spec.components[0], spec.components[1]
    f32 = np.float32
    dz = f32(src["target_dist"])
    z0 = ph["pos"][2] - 0.5 * ph["nz"] * ph["voxel"]   # entry face of the steps
    y_c = ph["pos"][1] + wl.staircase_step_y(6)         # lab y of step 6's centre
    checked = 0
    for i in range(n):
        if det[i] <= 0.0:
            continue
        sx, sy, E, tx, ty, w0 = (f32(st[r][i]) for r in range(6))
        dx, dy = f32(tx - sx), f32(ty - sy)
        ln = f32(np.sqrt(f32(f32(f32(dx * dx) + f32(dy * dy)) + f32(dz * dz))))
        il = f32(f32(1.0) / ln)
        k = np.array([f32(dx * il), f32(dy * il), f32(dz * il)], dtype=np.float64)
        y_in = float(sy) + k[1] / k[2] * z0
        y_out = float(sy) + k[1] / k[2] * (z0 + 0.026)
        if max(abs(y_in - y_c), abs(y_out - y_c)) > 9.5 * MM:
            continue
        mu = orc.mu(spec, 1, float(E), 32)
        assert det[i] == pytest.approx(float(w0) * math.exp(-mu * 0.026 / k[2]), rel=1e-9)
        checked += 1
    assert checked > n // 10
