"""The allocation-free batched trace (for callers that cannot allocate device
memory) gives the same monitors and tallies as the regular batched trace, on
two calls in a row, and allocates no device memory while doing so."""

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


def instruments(mcx, prec):
    specs = [wl.absorption_instrument(angle=0.4 * i, instr_id=i, nx=16, ne=16) for i in range(3)]
    specs += [wl.flat_slit_instrument(slit_w=w * MM, instr_id=3 + j) for j, w in enumerate((0.2, 1.5))]
    return specs, [mcx.Instrument(s, precision=prec) for s in specs]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_static_batch_matches_batch(env, prec):
    mcx, torch = env
    budgets = [300_001, 0, 77, 150_000, 99_999]
    specs, regular = instruments(mcx, prec)
    _, static = instruments(mcx, prec)
    b = mcx.Batch(regular, budgets, chunk_rays=1 << 14)
    for seed in (41, 42):                      # two calls in a row
        b.trace(seed)
        mcx.batch_trace_static(static, budgets, seed, chunk_rays=1 << 14)
    torch.cuda.synchronize()
    rtol = 1e-9 if prec == "fp64" else 1e-6
    for spec, x, y in zip(specs, static, regular):
        for c, comp in enumerate(spec.components):
            if not comp["type"].startswith("mon_"):
                continue
            a, r = x.monitor(c), y.monitor(c)
            assert (a[0] == r[0]).all()
            np.testing.assert_allclose(a[1], r[1], rtol=rtol, atol=0)
            np.testing.assert_allclose(a[2], r[2], rtol=2 * rtol, atol=0)
        ta, tr = x.tallies(), y.tallies()
        assert ta["n_emit"] == tr["n_emit"]
        np.testing.assert_allclose(ta["lost"], tr["lost"], rtol=rtol, atol=1e-9 * max(tr["sum_w0"], 1.0))
        assert ta["sum_wend"] == pytest.approx(tr["sum_wend"], rel=rtol, abs=1e-12)


def test_static_batch_allocates_nothing_and_checks_size(env):
    mcx, torch = env
    _, insts = instruments(mcx, "mixed")
    budgets = [50_000] * len(insts)
    mcx.batch_trace_static(insts, budgets, 7)   # first call: set-up on this device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for seed in (8, 9):
        mcx.batch_trace_static(insts, budgets, seed)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    with pytest.raises(mcx.McxError) as err:
        mcx.batch_trace_static([insts[0]] * 513, [1] * 513, 1)
    assert "at most 512" in str(err.value)
