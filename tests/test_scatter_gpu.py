"""Scattering in the voxel phantom on the GPU (the paper's step-wise march,
Sec. 3.3): monitors equal the oracle's in both forms, generic and compiled
(counts bit-exact: every decision - the scattering depth against its draw,
the fixed-point voxel, the new direction - is the oracle's), also for a dense
scatterer that reaches the eight-scattering limit, Rayleigh and Compton
events, energy-dependent coefficient tables (looked up again after each
Compton event), and in a batch; given starts are refused (the draws
continue the ray's own stream)."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

from test_parity_gpu import MODE, assert_parity, assert_parity_mixed_phantom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mcx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_08747_gb300 import build
    build.build()
    from paper_2410_08747_gb300 import mcx as m
    return m


def check(gpu, ref, spec, prec):
    if prec == "fp64":
        assert_parity(gpu, ref, spec, prec)
    else:
        assert_parity_mixed_phantom(gpu, ref, spec)


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("mu_s,compton,edep", [(20.0, 0.0, False), (300.0, 0.0, False), (20.0, 2.0, False),
                                               (20.0, 2.0, True)])
def test_scattering_phantom_parity(mcx, orc, prec, compiled, mu_s, compton, edep):
    """Rayleigh events alone, dense Rayleigh, Compton events twice as
    likely as Rayleigh ones (energies shift, absorption ahead re-looked-up),
    and the same with energy-dependent tables (Rayleigh ~ E^-2, Compton ~
    Klein-Nishina: the scattering ahead re-looked-up too)."""
    spec = wl.scatter_block(mu_s=mu_s, compton=compton, energy_dependent=edep)
    n = 40_000
    gpu = mcx.Instrument(spec, precision=prec, specialize=compiled)
    gpu.trace_range(0, n, 21)
    ref = orc.trace(spec, 0, n, 21, MODE[prec], threads=8)
    check(gpu, ref, spec, prec)
    N = gpu.monitor(2)[0]
    assert N.sum() > 0.05 * n


@pytest.mark.parametrize("edep", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_dense_scatterer_parity(mcx, orc, prec, edep):
    """mean free path 0.1 mm: every ray uses all eight scatterings (with
    energy-dependent tables: up to eight lookups at new energies)."""
    spec = wl.scatter_block(mu_s=5e3, absorb=False, compton=1.0, energy_dependent=edep)
    gpu = mcx.Instrument(spec, precision=prec)
    gpu.trace_range(0, 20_000, 5)
    ref = orc.trace(spec, 0, 20_000, 5, MODE[prec], threads=8)
    check(gpu, ref, spec, prec)


def test_scattering_in_a_batch_and_given_starts_refused(mcx):
    import torch
    specs = [wl.scatter_block(mu_s=50.0, instr_id=0), wl.scatter_block(mu_s=5.0, instr_id=1, seed=3)]
    alone = []
    for s in specs:
        g = mcx.Instrument(s, precision="mixed")
        g.trace(30_000, 8)
        alone.append(g)
    insts = [mcx.Instrument(s, precision="mixed") for s in specs]
    b = mcx.Batch(insts, [30_000, 30_000], chunk_rays=1 << 12)
    b.trace(8)
    for x, y in zip(insts, alone):
        assert (x.monitor(2)[0] == y.monitor(2)[0]).all()
        np.testing.assert_allclose(x.monitor(2)[1], y.monitor(2)[1], rtol=1e-6)
    st = torch.zeros(6 * 16, dtype=torch.float32, device="cuda")
    with pytest.raises(mcx.McxError):
        insts[0].trace_starts(st, 16)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_turned_rays_meet_an_analytic_absorber(mcx, orc, prec):
    """After a lens or a scattering phantom has turned the ray, an analytic
    absorber behind it sees the new line (in the mixed form its exact
    binary32 direction): monitors equal the oracle's."""
    foc = wl.focusing_instrument()
    foc.components.insert(2, wl.component("abs_box", pos=(0, 0, 31.6), wx=2e-4, wy=2e-4, wz=5e-3,
                                          material=0))
    blk = wl.scatter_block(mu_s=40.0)
    blk.components.insert(2, wl.component("abs_sphere", pos=(0.002, 0, 1.03), radius=0.01,
                                          material=1))
    for spec in (foc, blk):
        for compiled in (False, True):
            gpu = mcx.Instrument(spec, precision=prec, specialize=compiled)
            gpu.trace_range(0, 30_000, 19)
            ref = orc.trace(spec, 0, 30_000, 19, MODE[prec], threads=8)
            check(gpu, ref, spec, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_with_optics_and_scattering(mcx, prec):
    """A batch mixing the focusing instrument, a scattering block and the
    absorption instrument takes the kernel with every path, generic, by
    families and allocation-free, and equals each instrument alone."""
    import torch
    specs = [wl.focusing_instrument(instr_id=0),
             wl.scatter_block(mu_s=30.0, compton=1.0, instr_id=1, energy_dependent=True),
             wl.absorption_instrument(nx=16, ne=16, instr_id=2)]
    budgets = [40_000, 30_000, 20_000]
    rtol = 1e-9 if prec == "fp64" else 1e-6
    alone = []
    for s, b in zip(specs, budgets):
        g = mcx.Instrument(s, precision=prec)
        g.trace(b, 4)
        alone.append(g)
    for mode in ("generic", "families", "static"):
        insts = [mcx.Instrument(s, precision=prec) for s in specs]
        if mode == "static":
            mcx.batch_trace_static(insts, budgets, 4, chunk_rays=1 << 13)
            torch.cuda.synchronize()
        else:
            bt = mcx.Batch(insts, budgets, chunk_rays=1 << 13)
            if mode == "families":
                bt.specialize()
            bt.trace(4)
        for s, x, y in zip(specs, insts, alone):
            for c, comp in enumerate(s.components):
                if comp["type"].startswith("mon_"):
                    a, r = x.monitor(c), y.monitor(c)
                    assert (a[0] == r[0]).all(), (mode, c)
                    np.testing.assert_allclose(a[1], r[1], rtol=rtol, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_edxct_water_scatterer_parity(mcx, orc, prec):
    """The paper's EDXCT scanner with its water block scattering by water's
    energy-dependent tables on the 1/3-voxel march (the benchmark's
    scattering workload): the compiled kernel's monitors equal the
    oracle's."""
    spec = wl.edxct_scatter_instrument()
    n = 400_000      # ~1 % reach a line detector
    gpu = mcx.Instrument(spec, precision=prec, specialize=True)
    gpu.trace_range(10**10, 10**10 + n, 4)
    ref = orc.trace(spec, 10**10, 10**10 + n, 4, MODE[prec], threads=8)
    check(gpu, ref, spec, prec)


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_compton_step_table_parity(mcx, orc, prec, compiled):
    """Coefficients with a step on a cell boundary (Compton 50 /m above
    95 keV, 1 /m below): every lookup after a Compton event decides the
    steps ahead, and the monitors equal the oracle's."""
    from test_scatter import compton_step_block
    spec = compton_step_block()
    n = 40_000
    gpu = mcx.Instrument(spec, precision=prec, specialize=compiled)
    gpu.trace_range(0, n, 3)
    ref = orc.trace(spec, 0, n, 3, MODE[prec], threads=8)
    check(gpu, ref, spec, prec)
