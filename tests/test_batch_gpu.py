"""The batched persistent launch equals tracing each instrument alone (counts
bit-exact, sums to rounding), with and without graph replay, across chunk
sizes and after autotuning; seeds change between replays."""

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
    return m


def small_batch():
    specs = [wl.absorption_instrument(angle=0.3 * i, instr_id=i, nx=16, ne=16) for i in range(5)]
    specs += [wl.flat_slit_instrument(slit_w=w * MM, instr_id=5 + j) for j, w in enumerate((0.1, 0.5, 2.0))]
    budgets = [123_457, 0, 1, 33, 250_000, 77_777, 100_000, 64]
    return specs, budgets


def monitors(spec):
    return [i for i, c in enumerate(spec.components) if c["type"].startswith("mon_")]


def alone(mcx, spec, budget, seeds, prec):
    g = mcx.Instrument(spec, precision=prec)
    for s in seeds:
        g.trace(budget, s)
    return g


def assert_same(a, b, spec, rtol):
    for c in monitors(spec):
        x, y = a.monitor(c), b.monitor(c)
        assert (x[0] == y[0]).all()
        np.testing.assert_allclose(x[1], y[1], rtol=rtol, atol=0)
    ta, tb = a.tallies(), b.tallies()
    assert ta["n_emit"] == tb["n_emit"]
    np.testing.assert_allclose(ta["lost"], tb["lost"], rtol=rtol, atol=1e-9 * max(tb["sum_w0"], 1))
    assert ta["sum_w0"] == pytest.approx(tb["sum_w0"], rel=rtol, abs=1e-12)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("graph,chunk", [(True, 1 << 12), (False, 1 << 16), (True, 1 << 20)])
def test_batch_equals_alone(mcx, prec, graph, chunk):
    specs, budgets = small_batch()
    insts = [mcx.Instrument(s, precision=prec) for s in specs]
    b = mcx.Batch(insts, budgets, chunk_rays=chunk, use_graph=graph)
    assert b.items() == sum((bud + chunk - 1) // chunk for bud in budgets)
    b.trace(21)
    b.trace(22)            # a replay with a new seed
    b.synchronize()
    for spec, inst, bud in zip(specs, insts, budgets):
        ref = alone(mcx, spec, bud, (21, 22), prec)
        assert_same(inst, ref, spec, 1e-9 if prec == "fp64" else 1e-6)


def test_autotune_keeps_results(mcx):
    specs, budgets = small_batch()
    insts = [mcx.Instrument(s, precision="mixed") for s in specs]
    b = mcx.Batch(insts, budgets)
    chosen = b.autotune(20_000)
    assert chosen["block_size"] in (128, 256) and chosen["chunk_rays"] > 0
    assert chosen["use_graph"] == 1
    for inst in insts:                       # autotuning leaves clean monitors
        assert inst.tallies()["n_emit"] == 0
        assert all(inst.monitor(c)[0].sum() == 0 for c in monitors(inst.spec))
    b.trace(5)
    b.synchronize()
    for spec, inst, bud in zip(specs, insts, budgets):
        assert_same(inst, alone(mcx, spec, bud, (5,), "mixed"), spec, 1e-6)


def test_axisymmetric_projections_agree(mcx):
    """Rotating the cylinder about its own axis leaves every projection's
    expectation unchanged: the detector totals of 8 angles agree within
    their statistical errors."""
    n = 8
    specs = [wl.absorption_instrument(angle=2 * np.pi * i / n, instr_id=i, nx=16, ne=8) for i in range(n)]
    insts = [mcx.Instrument(s, precision="mixed") for s in specs]
    b = mcx.Batch(insts, [2_000_000] * n)
    b.trace(3)
    b.synchronize()
    m, s = [], []
    for inst in insts:
        N, sw, sw2 = inst.monitor(2)
        mean = sw.sum() / 2e6
        m.append(mean)
        s.append(np.sqrt((sw2.sum() / 2e6 - mean**2) / 2e6))
    m, s = np.array(m), np.array(s)
    z = (m - m.mean()) / s
    assert np.abs(z).max() < 5


def family_batch():
    """Three instrument families: rotated cylinders (angle 0 keeps the identity
    frame, so the frame flag varies too), slits of different widths, and
    rotated voxel phantoms."""
    specs = [wl.absorption_instrument(angle=0.4 * i, instr_id=i, nx=16, ne=16) for i in range(4)]
    specs += [wl.flat_slit_instrument(slit_w=w * MM, instr_id=4 + j) for j, w in enumerate((0.1, 0.5, 2.0))]
    specs += [wl.ct_instrument(angle=0.3 * k, n=16, voxel=8 * MM, n_pix=16, pix=16 * MM, ne=16,
                               window=1.5, instr_id=7 + k) for k in range(2)]
    budgets = [100_003, 0, 77, 60_000, 50_001, 1, 40_000, 30_007, 25_000]
    return specs, budgets


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_compiled_by_families_equals_generic(mcx, prec):
    """The batch kernel compiled by families (shared fields as constants, the
    varying ones read per instrument) traces every ray as the generic batch
    kernel does: counts bit-exact, sums to the rounding of the atomic order,
    through graph replays with changing seeds, and back to generic."""
    specs, budgets = family_batch()
    gen = [mcx.Instrument(s, precision=prec) for s in specs]
    fam = [mcx.Instrument(s, precision=prec) for s in specs]
    bg = mcx.Batch(gen, budgets, chunk_rays=1 << 14)
    bf = mcx.Batch(fam, budgets, chunk_rays=1 << 14)
    bf.specialize()
    for seed in (3, 4):
        bg.trace(seed)
        bf.trace(seed)
    rtol = 1e-9 if prec == "fp64" else 1e-6
    for spec, x, y in zip(specs, fam, gen):
        assert_same(x, y, spec, rtol)
    bf.specialize(False)              # the generic kernel again
    bf.trace(5)
    bg.trace(5)
    for spec, x, y in zip(specs, fam, gen):
        assert_same(x, y, spec, rtol)
    bf.close()
    bg.close()


def test_large_detectors_get_short_items(mcx):
    """An instrument with a 100 MB detector is cut into items of c rays, c the
    largest power of two with grid x c <= budget (at least 4096); an
    instrument with small monitors keeps chunk_rays; the results still equal
    each instrument traced alone."""
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    grid = n_sm * 2
    specs = [wl.absorption_instrument(instr_id=0),
             wl.flat_slit_instrument(slit_w=0.5 * MM, instr_id=1),
             wl.absorption_instrument(angle=0.4, instr_id=2)]
    budgets = [20_000_000, 300_000, 1_000_000]
    chunk = 1 << 18
    insts = [mcx.Instrument(s, precision="mixed") for s in specs]
    b = mcx.Batch(insts, budgets, chunk_rays=chunk, block_size=256, blocks_per_sm=2)

    def c_of(budget):
        p = 1
        while 2 * p <= budget // grid:
            p *= 2
        return min(chunk, max(p, 4096))

    want = [c_of(budgets[0]), chunk, c_of(budgets[2])]
    assert want[0] < chunk and want[2] == 4096
    assert b.items() == sum((bud + c - 1) // c for bud, c in zip(budgets, want))
    b.trace(5)
    b.synchronize()
    for spec, inst, bud in zip(specs, insts, budgets):
        ref = alone(mcx, spec, bud, (5,), "mixed")
        assert_same(inst, ref, spec, 1e-6)


def test_oversized_work_list_is_refused_before_it_is_built(mcx):
    """2^50 rays in 4096-ray items would be 2^38 work items: the plan counts
    them first and refuses (MCX_ERR_INVALID) without building the list."""
    inst = mcx.Instrument(wl.flat_slit_instrument(slit_w=0.5 * MM, instr_id=0), precision="mixed")
    with pytest.raises(mcx.McxError) as e:
        mcx.Batch([inst], [1 << 50], chunk_rays=1 << 12)
    assert e.value.status == -1 and "too many work items" in str(e.value)
