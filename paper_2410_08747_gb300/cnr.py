"""Contrast-to-noise ratio of the EDXCT test piece (Sec. 5.1).

The paper judges how many rays a line of its scanner needs by imaging a
steel staircase over a lead rod: two regions of the projection, ten lines
by ten pixels, one over steel alone and one over steel and lead, give per
energy bin

    CNR = |I_mat - I_ref| / sqrt(s_mat^2 + s_ref^2)

with I the mean flat-field-normalised intensity of a region and s the
standard deviation of that mean; a least-squares line fitted to the CNR
above an energy threshold must stay above 1 over the whole spectrum.  This
module is that analysis, on monitor sums read from the library (host-side
numpy; the tracing itself runs in the library's kernels)."""

import numpy as np


def normalised(sw_lines: np.ndarray, sw_flat: np.ndarray) -> np.ndarray:
    """Flat-field normalisation: I[l, p, e] = sw_lines[l, p, e] / sw_flat[p, e]
    for lines l, pixels p and energy bins e (NaN where the flat field got no
    weight)."""
    flat = np.asarray(sw_flat, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(flat > 0, np.asarray(sw_lines, dtype=np.float64) / flat, np.nan)


def region_stats(values: np.ndarray):
    """Mean and standard deviation of the mean, per energy bin, of a region's
    values [lines, pixels, bins]: the sample standard deviation (n - 1) over
    its lines x pixels, divided by sqrt(n)."""
    v = np.asarray(values, dtype=np.float64).reshape(-1, values.shape[-1])
    n = v.shape[0]
    mean = v.mean(axis=0)
    sd_mean = v.std(axis=0, ddof=1) / np.sqrt(n)
    return mean, sd_mean


def cnr(i_mat: np.ndarray, i_ref: np.ndarray) -> np.ndarray:
    """CNR per energy bin of two regions' normalised intensities."""
    m1, s1 = region_stats(i_mat)
    m2, s2 = region_stats(i_ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.abs(m1 - m2) / np.sqrt(s1 * s1 + s2 * s2)


def fit_above(e: np.ndarray, y: np.ndarray, e_from: float):
    """Least-squares line y = a + b e over the bins with e >= e_from and a
    finite y; returns (a, b)."""
    e = np.asarray(e, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    ok = (e >= e_from) & np.isfinite(y)
    if ok.sum() < 2:
        return float("nan"), float("nan")
    A = np.stack([np.ones(ok.sum()), e[ok]], axis=1)
    (a, b), *_ = np.linalg.lstsq(A, y[ok], rcond=None)
    return float(a), float(b)


def passes(a: float, b: float, e_lo: float, e_hi: float) -> bool:
    """The paper's criterion: the fitted line stays above 1 over [e_lo, e_hi]
    (a line's minimum over an interval is at an end)."""
    return bool(min(a + b * e_lo, a + b * e_hi) > 1.0)


def bin_centres(e_min: float, e_max: float, ne: int) -> np.ndarray:
    return e_min + (np.arange(ne) + 0.5) * (e_max - e_min) / ne


def study(sw: list, labels: list, pixels: slice, e_min: float = 20.0, e_max: float = 160.0,
          e_from: float = 80.0) -> dict:
    """The CNR study of one scan: sw[i] is line i's central-detector sums
    [pixels, bins]; labels[i] is "ref", "mat" or "flat".  Returns the CNR per
    bin, the fit above e_from and whether it passes over [e_min, e_max]."""
    flat = [s for s, l in zip(sw, labels) if l == "flat"]
    if len(flat) != 1:
        raise ValueError("one flat-field line is needed")
    ref = np.stack([s[pixels] for s, l in zip(sw, labels) if l == "ref"])
    mat = np.stack([s[pixels] for s, l in zip(sw, labels) if l == "mat"])
    f = flat[0][pixels]
    c = cnr(normalised(mat, f), normalised(ref, f))
    e = bin_centres(e_min, e_max, c.shape[-1])
    a, b = fit_above(e, c, e_from)
    return {"cnr": c, "e": e, "fit": (a, b), "passes": passes(a, b, e_min, e_max)}
