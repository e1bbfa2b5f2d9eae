"""Instrument compilation: the kernel specialised to one instrument's
component table (constants folded, run-time compiled) against the CPU oracle
with the same bars as the generic kernel, and against the generic kernel
itself (counts bit-exact, sums to rounding of the atomic order)."""

import time

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl
from test_parity_gpu import (MM, MODE, assert_parity, assert_parity_mixed_phantom,
                             every_component_instrument, monitors, small_ct)

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


def spec_run(mcx, spec, begin, end, seed, prec):
    g = mcx.Instrument(spec, precision=prec, specialize=True)
    g.trace_range(begin, end, seed)
    return g


INSTRUMENTS = {
    "flat_slit": (lambda: wl.flat_slit_instrument(), 200_000),
    "absorption_small": (lambda: wl.absorption_instrument(nx=32, ne=32), 100_000),
    "every_component": (every_component_instrument, 150_000),
    "disk_slit_narrow": (lambda: wl.flat_slit_instrument(slit_w=0.1 * MM), 100_000),
}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(INSTRUMENTS))
def test_specialised_parity(mcx, orc, name, prec):
    make, n = INSTRUMENTS[name]
    spec = make()
    gpu = spec_run(mcx, spec, 0, n, 5, prec)
    ref = orc.trace(spec, 0, n, 5, MODE[prec], threads=8)
    assert_parity(gpu, ref, spec, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_specialised_phantom_parity(mcx, orc, prec):
    spec = small_ct(angle=0.6, spot=10e-6)
    n = 40_000
    gpu = spec_run(mcx, spec, 0, n, 4, prec)
    ref = orc.trace(spec, 0, n, 4, MODE[prec], threads=8)
    if prec == "mixed":
        assert_parity_mixed_phantom(gpu, ref, spec)
    else:
        assert_parity(gpu, ref, spec, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_specialised_equals_generic_full_detector(mcx, prec):
    """The 128x128x256 absorption detector over 3e6 rays: the specialised and
    generic kernels agree bin for bin."""
    spec = wl.absorption_instrument()
    a = mcx.Instrument(spec, precision=prec)
    b = mcx.Instrument(spec, precision=prec, specialize=True)
    for g in (a, b):
        g.trace_range(5_000_000, 8_000_000, 3)
    Na, swa, sw2a = a.monitor(2)
    Nb, swb, sw2b = b.monitor(2)
    assert np.array_equal(Na, Nb) and int(Na.sum()) == 3_000_000
    np.testing.assert_allclose(swb, swa, rtol=1e-12, atol=0)
    np.testing.assert_allclose(sw2b, sw2a, rtol=1e-12, atol=0)
    ta, tb = a.tallies(), b.tallies()
    assert ta["n_emit"] == tb["n_emit"]
    assert tb["sum_w0"] == pytest.approx(ta["sum_w0"], rel=1e-12)
    np.testing.assert_allclose(tb["lost"], ta["lost"], rtol=1e-9, atol=1e-9)


def test_source_cache_and_switching_back(mcx):
    spec = wl.absorption_instrument(nx=16, ne=16)
    g = mcx.Instrument(spec, precision="mixed")
    src = g.kernel_source()
    assert "kComps[3]" in src and "mcx_spec_trace" in src and "0x1." in src
    t0 = time.perf_counter()
    g.specialize()
    first = time.perf_counter() - t0
    h = mcx.Instrument(spec, precision="mixed")
    t0 = time.perf_counter()
    h.specialize()                       # same table: the compiled kernel is reused
    assert time.perf_counter() - t0 < max(0.05, 0.5 * first)
    g.trace_range(0, 50_000, 1)
    g.specialize(False)                  # back to the generic kernel
    g.trace_range(50_000, 100_000, 1)
    ref = mcx.Instrument(spec, precision="mixed")
    ref.trace_range(0, 100_000, 1)
    assert np.array_equal(g.monitor(2)[0], ref.monitor(2)[0])
