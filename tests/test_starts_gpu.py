"""Ray-start buffers: the device sampler equals the oracle's binary32 starts
bit for bit; tracing given starts equals tracing the same rays directly and
equals the oracle's trace of those starts (counts bit-exact); the per-ray
detected weights equal the oracle's."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MM = 1e-3


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx
    return mcx, torch


SPECS = [
    lambda: wl.flat_slit_instrument(),
    lambda: wl.absorption_instrument(nx=32, ne=32),
    lambda: wl.ct_instrument(n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=32, window=1.5, spot=10e-6),
    lambda: wl.focusing_instrument(),
]


@pytest.mark.parametrize("k", range(len(SPECS)))
def test_starts_match_oracle_and_direct_trace(env, orc, k):
    mcx, torch = env
    spec = SPECS[k]()
    b, n, seed = 1_000_003, 30_001, 9
    st = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    g = mcx.Instrument(spec, precision="mixed")
    g.sample_starts(b, n, seed, st)
    ost = orc.sample_starts(spec, b, n, seed)
    gst = st.view(6, n).cpu().numpy()
    assert (gst[:5].view(np.uint32) == ost[:5].view(np.uint32)).all()
    # w0 is weight-only binary32 arithmetic: a Gaussian source's divergence
    # weight exp(-a^2/2) with a^2 up to ~14 carries ~1e-6 of the rounding of a
    np.testing.assert_allclose(gst[5], ost[5], rtol=1e-5 if k == 3 else 1e-6)
    det = torch.empty(n, dtype=torch.float32, device="cuda")
    g.trace_starts(st, n, b, det)
    direct = mcx.Instrument(spec, precision="mixed")
    direct.trace_range(b, b + n, seed)
    ref, odet = orc.trace_starts(spec, gst)
    mons = [i for i, c in enumerate(spec.components) if c["type"].startswith("mon_")]
    for c in mons:
        a, d, o = g.monitor(c), direct.monitor(c), ref.monitor(c)
        assert (a[0] == d[0]).all()
        assert (a[0].astype(np.int64) == o[0]).all()
        np.testing.assert_allclose(a[1], d[1], rtol=1e-6, atol=0)
    dd = det.cpu().numpy().astype(np.float64)
    assert (dd[odet == 0] == 0).all()          # not scored on either side
    scale = max(np.abs(odet).max(), 1e-30)
    np.testing.assert_allclose(dd, odet, rtol=1e-4, atol=1e-5 * scale)
