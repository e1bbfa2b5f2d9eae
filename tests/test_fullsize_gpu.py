"""Parity of the CUDA path with the CPU oracle where earlier tests were thin:

* the monitors' bin rule at bin edges (the exact-rational edge instruments of
  test_bin_edges): every edge case lands in the same bin on the GPU, in both
  forms, generic and compiled, as the rule says;
* the kernel compiled for the absorption instrument (the benchmark's kernel)
  on the full 128x128x256 detector, against the oracle in both modes;
* the full 256^3 CT phantom on a 2e5-ray slice that straddles the boundary
  between two 2^24-ray chunks of the walk's ray ordering (ids are traced in
  aim-tile order within a chunk), obtained as the difference of two GPU runs.
"""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl
from test_bin_edges import RAYS, edge_cases, edge_instrument, expected_counts
from test_parity_gpu import MODE, assert_parity, monitors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx as m
    m.lib()
    return m


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_edge_rays_bin_by_the_rule_on_the_gpu(mcx, prec):
    mode = MODE[prec]
    n = 0
    for kind, lo, hi, nb, v in edge_cases(mode):
        g = mcx.Instrument(edge_instrument(kind, lo, hi, nb, v), precision=prec)
        g.trace(RAYS, 1)
        got = g.monitor(1)[0].astype(np.int64)
        assert np.array_equal(got, expected_counts(kind, lo, hi, nb, v, mode, RAYS)), (kind, lo, hi, nb, v, got)
        g.close()
        n += 1
    assert n > 150


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_edge_rays_compiled_kernel(mcx, prec):
    """Compiled kernels fold the monitor's lo and inv into constants: the
    cases on and next to hi and to an inner edge of two monitors."""
    mode = MODE[prec]
    picked = []
    for mon in (("e", 10.1, 10.4, 3), ("psd_x", 0.1e-3, 0.7e-3, 3)):
        vals = [v for kind, lo, hi, nb, v in edge_cases(mode) if (kind, lo, hi, nb) == mon]
        inner = mon[1] + (mon[2] - mon[1]) / mon[3]
        for target in (inner, mon[2]):
            picked += [mon + (v,) for v in sorted(vals, key=lambda v: abs(v - target))[:3]]
    assert len(picked) >= 8
    for kind, lo, hi, nb, v in picked:
        g = mcx.Instrument(edge_instrument(kind, lo, hi, nb, v), precision=prec, specialize=True)
        g.trace(RAYS, 1)
        got = g.monitor(1)[0].astype(np.int64)
        assert np.array_equal(got, expected_counts(kind, lo, hi, nb, v, mode, RAYS)), (kind, lo, hi, nb, v, got)
        g.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_compiled_absorption_full_detector_vs_oracle(mcx, orc, prec):
    """The kernel compiled for the 128x128x256 absorption instrument (the
    benchmark's kernel, in its launch shape) on 60,001 rays far from id 0."""
    spec = wl.absorption_instrument()
    b, e = 7_654_321_000, 7_654_321_000 + 60_001
    g = mcx.Instrument(spec, precision=prec, specialize=True)
    g.trace_range(b, e, 2)
    ref = orc.trace(spec, b, e, 2, MODE[prec], threads=8)
    assert_parity(g, ref, spec, prec)


def _difference(a, b, spec):
    """Monitors of run a minus run b (a traced a superset of b's rays)."""
    out = {}
    for c in monitors(spec):
        Na, swa, sw2a = a.monitor(c)
        Nb, swb, sw2b = b.monitor(c)
        out[c] = (Na.astype(np.int64) - Nb.astype(np.int64), swa - swb, sw2a - sw2b)
    return out


class _Diff:
    def __init__(self, d):
        self.d = d

    def monitor(self, c):
        return self.d[c]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_ct_full_phantom_slice_across_order_chunks(mcx, orc, prec):
    """Run A traces [b, b + 2^24 + 1e5), two chunks of the ray ordering; run
    B traces [b, b + 2^24 - 1e5), inside A's first chunk.  A - B holds the
    2e5 rays around A's chunk boundary, the first half ordered within A's
    first chunk, the second half within its second; it must equal the oracle
    on those ids."""
    spec = wl.ct_instrument()
    chunk, half = 1 << 24, 100_000
    b = 333_000_000
    A = mcx.Instrument(spec, precision=prec)
    A.trace_range(b, b + chunk + half, 4)
    B = mcx.Instrument(spec, precision=prec)
    B.trace_range(b, b + chunk - half, 4)
    diff = _Diff(_difference(A, B, spec))
    ref = orc.trace(spec, b + chunk - half, b + chunk + half, 4, MODE[prec], threads=16)
    for c in monitors(spec):
        N, sw, sw2 = diff.monitor(c)
        No, swo, sw2o = ref.monitor(c)
        assert np.array_equal(N, No), f"monitor {c}: counts differ in {(N != No).sum()} bins"
        if prec == "fp64":
            # the two runs' sums carry 1e-16 of their own (larger) totals
            scale = np.maximum(np.abs(swo), A.monitor(c)[1] * 1e-6)
            assert np.all(np.abs(sw - swo) <= 1e-9 * scale + 1e-12), np.abs(sw - swo).max()
        else:
            assert abs(sw.sum() - swo.sum()) <= 1e-5 * swo.sum()
            mean = swo[swo > 0].mean()
            err = np.abs(sw - swo) / np.maximum(swo, mean)
            assert err.max() <= 3e-5, err.max()
    assert int(ref.monitor(monitors(spec)[0])[0].sum()) > 0.5 * 2 * half


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_monitor_total_equals_sum_of_bins(mcx, prec):
    spec = wl.absorption_instrument()
    g = mcx.Instrument(spec, precision=prec)
    g.trace_range(0, 2_000_003, 9)
    N, sw, sw2 = g.monitor(2)
    n, a, b = g.monitor_total(2)
    assert n == int(N.sum()) == 2_000_003
    assert a == pytest.approx(float(sw.sum()), rel=1e-12)
    assert b == pytest.approx(float(sw2.sum()), rel=1e-12)
    g.reset()
    assert g.monitor_total(2) == (0, 0.0, 0.0)
