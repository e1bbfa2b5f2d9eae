"""Exact-rational brute force of the monitors' bin rule at bin edges.

Monitors accumulate N, sum p and sum p^2 per bin (paper Sec. 2.2.2); the
paper prints no binning arithmetic, and the reading here is half-open bins
[lo, hi) with bin = floor((v - lo) * inv), inv = n / (hi - lo) formed once in
binary64 (rounded to binary32 in the binary32 decision type, with lo), and
values outside [lo, hi) dropped.  These tests fix that rule against two
things that are not the oracle:

* the mathematical bin floor((v - lo) n / (hi - lo)) in exact rationals
  (Python `fractions`): every ray farther than the rule's rounding bound from
  an edge lands in it;
* the rule's own operation sequence with each operation rounded exactly once
  (round-to-nearest-even of the exact rational result): rays on an edge and
  within a few ulp of it, and of hi, land where that sequence says.

Rays here are parallel to the optical axis from a point source placed at the
wanted coordinate, with a zero-width aim window and a zero-width energy band,
so every ray of an instrument reaches the monitor at exactly the chosen
coordinate and energy (2x2 and 3x1 position monitors, 3-bin energy monitors).
A second test draws 1e4 random energies through the draw contract and bins
them the same way.  A third compiles the oracle with each of three plausible
mistakes planted in its bin function and shows that the pin fails for each.
"""

from fractions import Fraction as F
import math

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

MM = 1e-3


# ------------------------------------------------------------------ exact rounding
def rn64(q: F) -> float:
    """q rounded to the nearest binary64 (ties to even): Python's int / int
    true division is correctly rounded."""
    return q.numerator / q.denominator


def rn32(q: F) -> float:
    """q rounded to the nearest binary32 (ties to even), as a Python float."""
    if q == 0:
        return 0.0
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if F(2) ** e > a:
        e -= 1
    e = max(e, -126)                     # subnormals: fixed quantum 2^-149
    m = round(a / F(2) ** (e - 23))      # Fraction rounding: half to even
    v = math.ldexp(float(m), e - 23)     # exact: m <= 2^24
    return v if q > 0 else -v


def test_rn32_matches_numpy_on_exact_doubles():
    """numpy's binary64 -> binary32 conversion is one correctly rounded step
    from an exactly represented value: the two roundings must agree."""
    rng = np.random.default_rng(11)
    xs = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-8, 8, 2000),
                         [1 + 2.0**-24, 1 + 3 * 2.0**-24, 1 - 2.0**-25, 0.1, 1e-3]])
    for x in xs:
        assert rn32(F(float(x))) == float(np.float32(x)), x


def contract_bin(v: float, lo: float, hi: float, n: int, mode: int) -> int:
    """The monitor's bin rule, each operation rounded once in the decision
    type: 64 -> binary64 throughout; 32 -> inv and lo rounded to binary32,
    then the difference and the product in binary32."""
    if mode == 64:
        inv = rn64(F(n) / F(rn64(F(hi) - F(lo))))
        d = rn64(F(v) - F(lo))
        f = rn64(F(d) * F(inv))
    else:
        inv = rn32(F(rn64(F(n) / F(rn64(F(hi) - F(lo))))))
        d = rn32(F(rn32(F(v))) - F(rn32(F(lo))))
        f = rn32(F(d) * F(inv))
    if not (f >= 0.0 and f < n):
        return -1
    return int(math.floor(f))


def exact_bin(v: float, lo: float, hi: float, n: int) -> int:
    """The mathematical half-open bin of v, in exact rationals."""
    V, L, H = F(v), F(lo), F(hi)
    if not (L <= V < H):
        return -1
    return int(math.floor((V - L) * n / (H - L)))


def rounding_bound(lo: float, hi: float, mode: int) -> float:
    """Distance from an edge inside which the rule's roundings (of hi - lo,
    of n / that, of lo in binary32, of v - lo and of the product) can move a
    value across it: a few unit roundoffs of the range's magnitude."""
    u = 2.0**-53 if mode == 64 else 2.0**-24
    return 8 * u * (abs(hi - lo) + abs(lo) + abs(hi))


def near(v: float, mode: int, k: int) -> float:
    """The value k ulps of the decision type above (k > 0) or below v."""
    if mode == 64:
        x = np.float64(v)
        step = np.float64(np.inf if k > 0 else -np.inf)
    else:
        x = np.float32(v)
        step = np.float32(np.inf if k > 0 else -np.inf)
    for _ in range(abs(k)):
        x = np.nextafter(x, step)
    return float(x)


def edge_values(lo: float, hi: float, n: int, mode: int, span: int = 4):
    """Coordinates on every bin edge lo + j (hi - lo)/n (rounded to the
    decision type), k = -span..span ulps around each, and hi itself."""
    out = []
    for j in range(n + 1):
        e = F(lo) + j * (F(hi) - F(lo)) / n
        base = rn64(e) if mode == 64 else rn32(e)
        out += [near(base, mode, k) for k in range(-span, span + 1)]
    out += [hi, near(hi, mode, -1), near(hi, mode, 1)]
    return sorted(set(out))


# ------------------------------------------------------------------ instruments
def _point_source(x: float, y: float, E: float):
    return wl.component("source", pos=(x, y, 0.0), shape="point", spectrum="flat", e_min=E, e_max=E,
                        target_dist=1.0, target_w=0.0, target_h=0.0)


# (kind, lo, hi, n): 2x2 and 3x1 position monitors (x axis; the other axis
# sits in the middle of its first bin) and 3-bin energy monitors.  Edges that
# are not binary fractions (0.1 mm steps, 0.1 keV steps) and a range whose
# inverse width rounds (30 keV over 3 bins: inv = RN(0.1)).
MONITORS = [
    ("psd_x", -1 * MM, 1 * MM, 2),
    ("psd_y", -1 * MM, 1 * MM, 2),
    ("psd_x", 0.1 * MM, 0.7 * MM, 3),
    ("psd_x", -0.3 * MM, 0.9 * MM, 3),
    ("e", 10.1, 10.4, 3),
    ("e", 10.0, 40.0, 3),
    ("e", 20.0, 120.0, 3),
]


def edge_instrument(kind: str, lo: float, hi: float, n: int, v: float):
    """One instrument whose every ray meets the monitor at coordinate v."""
    if kind == "e":
        src = _point_source(0.0, 0.0, v)
        mon = wl.component("mon_e", pos=(0.0, 0.0, 1.0), ne=n, e_min=lo, e_max=hi,
                           xmin=-1 * MM, xmax=1 * MM, ymin=-1 * MM, ymax=1 * MM)
    elif kind == "psd_x":
        src = _point_source(v, -0.5 * MM, 15.0)
        mon = wl.component("mon_psd", pos=(0.0, 0.0, 1.0), nx=n, ny=2, xmin=lo, xmax=hi,
                           ymin=-1 * MM, ymax=1 * MM)
    else:
        src = _point_source(-0.5 * MM, v, 15.0)
        mon = wl.component("mon_psd", pos=(0.0, 0.0, 1.0), nx=2, ny=n, xmin=-1 * MM, xmax=1 * MM,
                           ymin=lo, ymax=hi)
    return wl.Instrument(components=[src, mon], name=f"edge_{kind}")


def expected_counts(kind: str, lo: float, hi: float, n: int, v: float, mode: int, rays: int,
                    rule=contract_bin):
    """Monitor counts the rule predicts for `rays` rays at coordinate v."""
    if kind == "e":
        nb, b = n, rule(v, lo, hi, n, mode)
    else:
        # the other axis: -0.5 mm, the middle of bin 0 of [-1, 1) mm over 2 bins
        assert contract_bin(-0.5 * MM, -1 * MM, 1 * MM, 2, mode) == 0
        i = rule(v, lo, hi, n, mode)
        nb = 2 * n
        # bin index iy * nx + ix: psd_x has nx = n, iy = 0; psd_y has nx = 2, ix = 0
        b = -1 if i < 0 else (i if kind == "psd_x" else 2 * i)
    N = np.zeros(nb, dtype=np.int64)
    if b >= 0:
        N[b] = rays
    return N


def edge_cases(mode: int):
    for kind, lo, hi, n in MONITORS:
        for v in edge_values(lo, hi, n, mode):
            yield kind, lo, hi, n, v


RAYS = 3


def _run_cases(orc, mode, lib_=None):
    """(case, oracle counts) for every edge case of `mode`."""
    out = []
    for kind, lo, hi, n, v in edge_cases(mode):
        r = orc.trace(edge_instrument(kind, lo, hi, n, v), 0, RAYS, 1, mode, lib_=lib_)
        out.append(((kind, lo, hi, n, v), r.monitor(1)[0].copy()))
    return out


@pytest.mark.parametrize("mode", [64, 32])
def test_edge_rays_follow_the_rule_and_the_exact_bin(orc, mode):
    n_cases = n_disagree = 0
    for (kind, lo, hi, n, v), N in _run_cases(orc, mode):
        n_cases += 1
        assert np.array_equal(N, expected_counts(kind, lo, hi, n, v, mode, RAYS)), (kind, lo, hi, n, v, N)
        # against the exact bin: equal unless v lies within the rounding bound of an edge
        vv = v if mode == 64 else rn32(F(v))
        rule = contract_bin(v, lo, hi, n, mode)
        exact = exact_bin(vv, lo, hi, n)
        if rule != exact:
            n_disagree += 1
            dist = min(abs(F(vv) - (F(lo) + j * (F(hi) - F(lo)) / n)) for j in range(n + 1))
            assert dist <= F(rounding_bound(lo, hi, mode)), (kind, lo, hi, n, v, rule, exact, float(dist))
    assert n_cases > 150
    # rays on and next to edges do cross: the bound is exercised, not vacuous
    assert 0 < n_disagree < n_cases // 2


@pytest.mark.parametrize("mode", [64, 32])
def test_random_energies_bin_exactly(orc, mode):
    """1e4 rays of a flat 10.1-10.4 keV source into a 3-bin energy monitor
    over the same band: each ray's energy from the draw contract
    (E = e_min + (e_max - e_min) u, u the ray's third draw, each operation
    rounded once), its bin by the rule; the histogram equals the oracle's
    counts bit for bit, and the exact rational bin of every ray agrees."""
    lo, hi, n, rays, seed = 10.1, 10.4, 3, 10_000, 9
    src = wl.component("source", shape="point", spectrum="flat", e_min=lo, e_max=hi,
                       target_dist=1.0, target_w=0.2 * MM, target_h=0.2 * MM)
    mon = wl.component("mon_e", pos=(0.0, 0.0, 1.0), ne=n, e_min=lo, e_max=hi,
                       xmin=-1 * MM, xmax=1 * MM, ymin=-1 * MM, ymax=1 * MM)
    inst = wl.Instrument(components=[src, mon], name="edge_random_e")
    r = orc.trace(inst, 0, rays, seed, mode)
    want = np.zeros(n, dtype=np.int64)
    for i in range(rays):
        if mode == 64:
            u = orc.uniform64(i, 0, seed, 2)
            E = rn64(F(lo) + F(rn64(F(rn64(F(hi) - F(lo))) * F(u))))
        else:
            u = float(orc.uniform32(i, 0, seed, 2))
            lo32, hi32 = rn32(F(lo)), rn32(F(hi))
            E = rn32(F(lo32) + F(rn32(F(rn32(F(hi32) - F(lo32))) * F(u))))
        b = contract_bin(E, lo, hi, n, mode)
        assert b == exact_bin(E, lo, hi, n) or b == -1 and E >= hi
        if b >= 0:
            want[b] += 1
    assert np.array_equal(r.monitor(1)[0], want)
    assert want.sum() == rays


# ------------------------------------------------------------------ planted mistakes
_BIN_INV = "const REAL inv = (REAL)((double)n / (hi - lo));"
_BIN_F = "const REAL f = (v - (REAL)lo) * inv;"
_BIN_TEST = "if (!(f >= (REAL)0) || !(f < (REAL)n)) return -1;\n  return (int)f;"
PLANTS = {
    # inv formed in binary32 even in the binary64 mode
    "inv_binary32": [("orc_core.inc", _BIN_INV, "const REAL inv = (REAL)((float)n / (float)(hi - lo));")],
    # a division by the bin width in place of the product with inv
    "divide_by_width": [("orc_core.inc", _BIN_F, "const REAL f = (v - (REAL)lo) / (REAL)((hi - lo) / n);")],
    # the last bin closed at hi
    "closed_at_hi": [("orc_core.inc", _BIN_TEST,
                      "if (!(f >= (REAL)0) || !(f <= (REAL)n)) return -1;\n  return f == (REAL)n ? n - 1 : (int)f;")],
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_each_planted_bin_mistake_fails_the_pin(orc, plant, tmp_path):
    L = orc.build_variant(PLANTS[plant], str(tmp_path / plant))
    caught = 0
    for mode in (64, 32):
        for (kind, lo, hi, n, v), N in _run_cases(orc, mode, lib_=L):
            if not np.array_equal(N, expected_counts(kind, lo, hi, n, v, mode, RAYS)):
                caught += 1
    assert caught > 0, f"the planted mistake {plant!r} passes the bin-edge pin"
