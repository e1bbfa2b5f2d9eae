"""Failures made on the host, seen through the C ABI: an allocation hook that
refuses the k-th request makes mcx_instrument_create (and the first monitor
read) return MCX_ERR_OOM, with every earlier allocation handed back and the
device still usable; bad launch arguments are refused before any launch."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
MM = 1e-3


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


def failing_allocator(mcx, fail_at):
    class A(mcx._TorchAllocator):
        def __init__(self):
            super().__init__(0)
            self.calls = 0
            self.frees = 0

        def _alloc(self, nbytes, ctx):
            k = self.calls
            self.calls += 1
            if k == fail_at:
                return None
            return super()._alloc(nbytes, ctx)

        def _free(self, ptr, ctx):
            self.frees += 1
            super()._free(ptr, ctx)
    return A()


def small_ct():
    return wl.ct_instrument(n=16, voxel=8 * MM, n_pix=16, pix=16 * MM, ne=16)


def small_scatter():
    return wl.scatter_block(nx=8, ny=8, nz=8, mu_s=30.0, compton=1.0)


@pytest.mark.parametrize("make", [small_ct, small_scatter, lambda: wl.focusing_instrument()])
def test_create_oom_at_every_allocation_releases_everything(mcx, make):
    spec = make()
    ok = failing_allocator(mcx, -1)
    g = mcx.Instrument(spec, precision="mixed", allocator=ok)
    n_allocs = ok.calls
    assert n_allocs >= 4                   # table, bins, tallies, mu tables (, phantom, ...)
    g.close()
    assert ok.frees == n_allocs and not ok.live
    for k in range(n_allocs):
        a = failing_allocator(mcx, k)
        with pytest.raises(mcx.McxError, match="OOM"):
            mcx.Instrument(spec, precision="mixed", allocator=a)
        assert a.calls >= k + 1
        assert not a.live, f"allocation {k}: {len(a.live)} buffers not returned"
    # the device is still usable afterwards
    g = mcx.Instrument(spec, precision="mixed")
    g.trace_range(0, 10_000, 1)
    mon = next(i for i, c in enumerate(spec.components) if c["type"].startswith("mon_"))
    assert int(g.monitor(mon)[0].sum()) > 0


def test_readout_scratch_oom_then_recovers(mcx):
    spec = small_ct()
    probe = failing_allocator(mcx, -1)
    g0 = mcx.Instrument(spec, precision="mixed", allocator=probe)
    n_create = probe.calls
    g0.close()
    a = failing_allocator(mcx, n_create)   # the first read's scratch
    g = mcx.Instrument(spec, precision="mixed", allocator=a)
    g.trace_range(0, 20_000, 3)
    with pytest.raises(mcx.McxError, match="OOM"):
        g.monitor(2)
    N, sw, _ = g.monitor(2)                # the next read allocates and succeeds
    ref = mcx.Instrument(spec, precision="mixed")
    ref.trace_range(0, 20_000, 3)
    assert np.array_equal(N, ref.monitor(2)[0])
    g.close()
    assert not a.live


def test_invalid_launch_arguments(mcx):
    spec = wl.flat_slit_instrument()
    g = mcx.Instrument(spec, precision="mixed")
    L = mcx.lib()
    assert L.mcx_trace_range(g._h, 10, 5, 1) == -1          # end < begin
    assert L.mcx_monitor_read(g._h, 0, None, None, None, 1) == -1   # not a monitor
    nb = g.monitor_bins(2)
    buf = np.zeros(nb + 1, dtype=np.float64)
    assert L.mcx_monitor_read(g._h, 2, None, buf.ctypes.data, None, nb + 1) == -1  # wrong size
    assert g.tallies()["n_emit"] == 0


def test_tensor_core_wait_that_runs_out_is_reported(mcx):
    """A bounded tensor-core wait made to run out (the test-only wait limit
    0: give up at once, then drain the MMAs in flight before freeing tensor
    memory) is reported as MCX_ERR_TIMEOUT, by the next sample call for the
    sampler and by the call itself for the forward pass and for training
    (whose weight-gradient products also drain their TMA loads); no device
    fault, and the device stays usable."""
    import torch
    spec = small_ct()
    src = spec.components[0]
    theta = wl.proposal_init(0).astype(np.float32)

    def proposal():
        return mcx.Proposal(0.2, 0.5 * src["target_w"], 0.5 * src["target_h"], [0.0] * 4, [1.0] * 4,
                            params=theta)

    inst = mcx.Instrument(spec, precision="mixed")
    n = 5_000
    buf = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    p = proposal()
    p.set_wait_limit(0)
    p.sample(inst, 0, n, 1, buf)            # queued; every wait gives up at once
    with pytest.raises(mcx.McxError) as err:
        p.sample(inst, 0, n, 1, buf)
    assert err.value.status == -4
    q = proposal()
    q.set_wait_limit(0)
    x = torch.zeros((256, 4), dtype=torch.float32, device="cuda")
    out = torch.empty((256, 40), dtype=torch.float32, device="cuda")
    with pytest.raises(mcx.McxError) as err:
        q.forward(x, out)
    assert err.value.status == -4
    # a training step: its tile kernel's waits and the weight-gradient
    # products' waits on their TMA loads give up at once, drain and report
    t = proposal()
    t.set_wait_limit(0)
    nh = 1000
    hist = torch.empty(6 * nh, dtype=torch.float32, device="cuda")
    inst.sample_starts(0, nh, 3, hist)
    det = torch.ones(nh, dtype=torch.float32, device="cuda")
    with pytest.raises(mcx.McxError) as err:
        t.train(hist, det, nh, batch=512)
    assert err.value.status == -4
    # the device still works: fresh proposals sample identical, finite starts
    b1 = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    b2 = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    proposal().sample(inst, 0, n, 1, b1)
    r = proposal()
    r.set_wait_limit(-1)                    # the default limit
    r.sample(inst, 0, n, 1, b2)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2) and bool(torch.isfinite(b1).all())
    inst.trace_range(0, 10_000, 2)
    assert int(inst.monitor(2)[0].sum()) > 0
