"""The mixed form's error against the binary64 form, per monitor.

The two forms draw their uniforms differently (binary32 draw j is the top 24
bits of Philox word j mod 4 of block j/4; binary64 draw j takes 53 bits of a
word pair of block j/2), so ray i of one form is not ray i of the other: the
two traces of the same ids are two samples of the same estimator.  The
precision change is an error only if it moves the expectation.  Per monitor:
* against the binary64 oracle on 4e5 rays: the difference of the total
  weights, in units of its standard deviation (both samples' variances from
  their sums of squared weights), |z| < 4; chi^2 per degree of freedom of the
  per-bin sums against the per-bin variances within 0.1 of 1;
* against the binary64 GPU form (itself equal to the oracle to 1e-9) on 1e8
  rays (2e7 behind the phantom), which bounds a bias 15x tighter: |z| < 4.
The two samples of each comparison use different seeds, so they are
independent and the variance of their difference is the sum of theirs.
The measured relative differences are printed (pytest -s)."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl
from test_parity_gpu import monitors, small_ct

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


CASES = {
    "flat_slit": (lambda: wl.flat_slit_instrument(), 400_000, 100_000_000),
    "absorption_64x64x64": (lambda: wl.absorption_instrument(nx=64, ne=64), 400_000, 100_000_000),
    "ct_32": (lambda: small_ct(spot=10e-6), 100_000, 20_000_000),
    "focusing_crl16": (lambda: wl.focusing_instrument(), 400_000, 100_000_000),
}


def _compare(N, sw, sw2, n, No, swo, sw2o, no):
    """z of the difference of the two mean weights per ray, chi^2/dof of the
    per-bin means, relative difference of the totals."""
    m, mo = float(sw.sum()) / n, float(swo.sum()) / no
    var = (float(sw2.sum()) / n - m * m) / n
    varo = (float(sw2o.sum()) / no - mo * mo) / no
    z = (m - mo) / np.sqrt(var + varo)
    vb = sw2 / (n * n) + sw2o / (no * no)
    used = vb > 0
    chi2 = float((((sw / n - swo / no)[used]) ** 2 / vb[used]).sum()) / max(int(used.sum()), 1)
    return z, chi2, (m - mo) / mo, int(used.sum())


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_form_against_binary64(mcx, orc, name):
    make, n, n_big = CASES[name]
    spec = make()
    b = 3_000_000
    g = mcx.Instrument(spec, precision="mixed")
    g.trace_range(b, b + n, 11)
    ref = orc.trace(spec, b, b + n, 14, 64, threads=16)       # another seed: independent samples
    big = mcx.Instrument(spec, precision="mixed")
    big.trace_range(10**9, 10**9 + n_big, 12)
    big64 = mcx.Instrument(spec, precision="fp64")
    big64.trace_range(10**9, 10**9 + n_big, 13)
    for c in monitors(spec):
        N, sw, sw2 = g.monitor(c)
        No, swo, sw2o = ref.monitor(c)
        if float(swo.sum()) <= 0:
            continue
        z, chi2, rel, dof = _compare(N, sw, sw2, n, No, swo, sw2o, n)
        Nb, swb, sw2b = big.monitor(c)
        Nd, swd, sw2d = big64.monitor(c)
        zb, chi2b, relb, dofb = _compare(Nb, swb, sw2b, n_big, Nd, swd, sw2d, n_big)
        print(f"{name} monitor {c}: vs oracle (4e5): rel {rel:+.2e} z {z:+.2f} chi2/dof {chi2:.3f} ({dof} bins); "
              f"vs GPU binary64 ({n_big:.0e}): rel {relb:+.2e} z {zb:+.2f} chi2/dof {chi2b:.3f}")
        assert abs(z) < 4, (c, z)
        if dof >= 1000:
            assert abs(chi2 - 1.0) < 0.1, (c, chi2)
        assert abs(zb) < 4, (c, zb)
