"""The fixed-step phantom traversal (Sec. 3.3: steps of voxel/s, each
weighted by the voxel at its end point) on the GPU: monitors equal the
oracle's in both forms, generic and compiled kernels (counts bit-exact, sums
within each form's bound); each ray's detected weight equals the oracle's to
binary32 rounding, which a single voxel sampled differently would break
(one 1/3-voxel step of water moves a weight by several percent); batches
that mix marching and walking instruments equal each instrument traced
alone."""

import numpy as np
import pytest

from paper_2410_08747_gb300 import workloads as wl

from test_parity_gpu import MODE, assert_parity, assert_parity_mixed_phantom, monitors

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


def marched_edxct(s=3.0, n_det=5, seed=4, instr_id=0):
    """The EDXCT scanner at 10 mm voxels with a random vacuum / water block
    (every step can change material), marched at s steps per voxel."""
    rng = np.random.default_rng(seed)
    vox = rng.integers(0, 2, size=(25, 35, 8)).astype(np.uint8)
    spec = wl.edxct_instrument(nx=8, ny=35, nz=25, voxel=10 * MM, n_det=n_det, det_px=32,
                               pix=3.2 * MM, ne=16, phantom=vox, instr_id=instr_id)
    spec.components[1]["march"] = s
    return spec


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_edxct_march_parity(env, orc, prec, compiled):
    """The paper's EDXCT block at full size (350 x 250 x 100 voxels of
    1 mm, ~750 steps of 1/3 mm per ray): the mixed form's optical depth,
    summed over so many equal steps, stays within the phantom bound."""
    mcx, _ = env
    spec = wl.edxct_instrument()
    spec.components[1]["march"] = 3
    n = 100_000
    gpu = mcx.Instrument(spec, precision=prec, specialize=compiled)
    gpu.trace_range(10**9, 10**9 + n, 4)
    ref = orc.trace(spec, 10**9, 10**9 + n, 4, MODE[prec], threads=8)
    if prec == "mixed":
        assert_parity_mixed_phantom(gpu, ref, spec)
    else:
        assert_parity(gpu, ref, spec, prec)


@pytest.mark.parametrize("compiled", [False, True])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("s", [3.0, 1.0, 7.5])
def test_march_parity(env, orc, prec, compiled, s):
    mcx, _ = env
    spec = marched_edxct(s)
    n = 50_000
    gpu = mcx.Instrument(spec, precision=prec, specialize=compiled)
    gpu.trace_range(0, n, 9)
    ref = orc.trace(spec, 0, n, 9, MODE[prec], threads=8)
    if prec == "mixed":
        assert_parity_mixed_phantom(gpu, ref, spec)
    else:
        assert_parity(gpu, ref, spec, prec)
    assert sum(int(gpu.monitor(c)[0].sum()) for c in monitors(spec)) > 0.9 * n


@pytest.mark.parametrize("compiled", [False, True])
def test_march_per_ray_weights(env, orc, compiled):
    mcx, torch = env
    spec = marched_edxct(3.0, n_det=1)
    b, n, seed = 77, 40_000, 5
    st = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    g = mcx.Instrument(spec, precision="mixed", specialize=compiled)
    g.sample_starts(b, n, seed, st)
    det = torch.empty(n, dtype=torch.float32, device="cuda")
    g.trace_starts(st, n, b, det)
    ref, odet = orc.trace_starts(spec, st.view(6, n).cpu().numpy())
    dd = det.cpu().numpy().astype(np.float64)
    assert (odet > 0).sum() > n // 2
    assert (dd[odet == 0] == 0).all()
    np.testing.assert_allclose(dd, odet, rtol=1e-4, atol=1e-6 * odet.max())


def test_march_approaches_the_walk(env):
    """Ray by ray, the march's optical depth differs from the exact walk's
    only at crossed faces, by at most a step each: on the same starts, the
    mean |tau_march - tau_walk| shrinks as the steps do, and the detected
    rays are the same."""
    mcx, torch = env
    n = 40_000
    walk = mcx.Instrument(marched_edxct(0.0, n_det=1), precision="mixed")
    st = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    walk.sample_starts(0, n, 3, st)
    dw = torch.empty(n, dtype=torch.float32, device="cuda")
    walk.trace_starts(st, n, 0, dw)
    dw = dw.cpu().numpy().astype(np.float64)
    gaps = []
    for s in (1.0, 3.0, 12.0):
        g = mcx.Instrument(marched_edxct(s, n_det=1), precision="mixed")
        dm = torch.empty(n, dtype=torch.float32, device="cuda")
        g.trace_starts(st, n, 0, dm)
        dm = dm.cpu().numpy().astype(np.float64)
        assert ((dm > 0) == (dw > 0)).all()
        ok = (dw > 1e-30) & (dm > 1e-30)
        gaps.append(float(np.abs(np.log(dm[ok]) - np.log(dw[ok])).mean()))
    assert gaps[0] > gaps[1] > gaps[2] > 0.0, gaps


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_mixing_march_and_walk(env, prec):
    mcx, torch = env
    specs = [marched_edxct(3.0, instr_id=0), marched_edxct(0.0, instr_id=1),
             marched_edxct(3.0, seed=8, instr_id=2), wl.absorption_instrument(nx=16, ne=16, instr_id=3)]
    budgets = [60_001, 40_000, 0, 30_000]
    rtol = 1e-9 if prec == "fp64" else 1e-6
    alone = []
    for spec, bud in zip(specs, budgets):
        g = mcx.Instrument(spec, precision=prec)
        g.trace(bud, 11)
        alone.append(g)
    for mode in ("generic", "families", "static"):
        insts = [mcx.Instrument(s, precision=prec) for s in specs]
        if mode == "static":
            mcx.batch_trace_static(insts, budgets, 11, chunk_rays=1 << 14)
            torch.cuda.synchronize()
        else:
            b = mcx.Batch(insts, budgets, chunk_rays=1 << 14)
            if mode == "families":
                b.specialize()
            b.trace(11)
        for spec, x, y in zip(specs, insts, alone):
            for c in monitors(spec):
                a, r = x.monitor(c), y.monitor(c)
                assert (a[0] == r[0]).all(), mode
                np.testing.assert_allclose(a[1], r[1], rtol=rtol, atol=0)
