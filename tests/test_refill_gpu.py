"""Refilled lanes on a scattering phantom (mixed form, Sec. 3.3: the
step-wise march in which a step may scatter the ray).  A lane takes its
next ray as soon as its ray is done, so lanes stand at different components
and steps; each ray must still take the one-ray trace's operations in the
same order.  Checked against the oracle (counts bit-exact, weights within the
mixed form's phantom bound, tallies within the same bound) and against the
batch kernel, which keeps one ray per lane (counts equal):

* a slit before the phantom that stops some rays before they reach it;
* a source window wider than the block, so some rays miss the grid;
* an analytic absorber and two monitors after the phantom;
* ranges of 1 ray, 45 rays and a ragged 30,011 rays far from id 0;
* 64- and 256-thread blocks, generic and compiled kernels."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

from test_parity_gpu import MODE, assert_parity_mixed_phantom

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


def refill_block(instr_id: int = 0) -> wl.Instrument:
    """The scattering block with a 60 mm source window (the block is 40 mm
    wide), a 50 x 30 mm slit before it, an absorbing sphere and a position
    and an energy monitor after it."""
    spec = wl.scatter_block(mu_s=40.0, compton=1.0, energy_dependent=True, instr_id=instr_id)
    src = spec.components[0]
    src["target_w"] = src["target_h"] = 60 * MM
    spec.components.insert(1, wl.component("slit_rect", pos=(0, 0, 0.95), xmin=-25 * MM, xmax=25 * MM,
                                           ymin=-15 * MM, ymax=15 * MM))
    spec.components.insert(3, wl.component("abs_sphere", pos=(0.004, 0, 1.035), radius=0.012,
                                           material=1))
    spec.components.append(wl.component("mon_e", pos=(0, 0, 1.2), ne=64, e_min=30.0, e_max=90.0,
                                        xmin=-0.1, xmax=0.1, ymin=-0.1, ymax=0.1))
    return spec


def check_tallies(gpu, ref, tol=3e-5):
    t = gpu.tallies()
    assert t["n_emit"] == ref.n_emit
    scale = max(ref.sum_w0, 1.0)
    assert abs(t["sum_w0"] - ref.sum_w0) <= 1e-6 * scale
    assert abs(t["sum_wend"] - ref.sum_wend) <= tol * scale
    np.testing.assert_allclose(t["lost"], ref.lost, rtol=tol, atol=tol * scale)


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("block", [64, 256])
@pytest.mark.parametrize("begin,n", [(0, 1), (7, 45), (3_000_000_019, 30_011)])
def test_refill_parity(mcx, orc, compiled, block, begin, n):
    spec = refill_block()
    gpu = mcx.Instrument(spec, precision="mixed", block_size=block, specialize=compiled)
    gpu.trace_range(begin, begin + n, 13)
    ref = orc.trace(spec, begin, begin + n, 13, MODE["mixed"], threads=8)
    assert_parity_mixed_phantom(gpu, ref, spec)
    check_tallies(gpu, ref)
    if n > 1000:
        # every kind of ray occurred: stopped by the slit, missed the grid,
        # scattered, reached the last monitor
        lost = ref.lost
        assert lost[1] > 0 and ref.monitor(len(spec.components) - 1)[0].sum() > 0


def test_refill_equals_one_ray_per_lane(mcx):
    """The batch kernel traces one ray per lane from start to end; the
    refilling kernel gives every monitor the same counts and sums to 1e-6."""
    spec = refill_block()
    alone = mcx.Instrument(spec, precision="mixed", specialize=True)
    alone.trace(200_000, 29)
    inst = mcx.Instrument(spec, precision="mixed")
    b = mcx.Batch([inst], [200_000], chunk_rays=1 << 14)
    b.trace(29)
    for c, comp in enumerate(spec.components):
        if comp["type"].startswith("mon_"):
            x, y = inst.monitor(c), alone.monitor(c)
            assert (x[0] == y[0]).all(), c
            np.testing.assert_allclose(x[1], y[1], rtol=1e-6, atol=0)
    np.testing.assert_allclose(inst.tallies()["lost"], alone.tallies()["lost"], rtol=1e-6, atol=1e-9)
