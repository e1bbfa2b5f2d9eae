"""The learned proposal on the GPU against the FP64 oracle (oracle/mlp.py):
network outputs and gradients with BF16-rounded operands mirrored, sampled
aim points and importance weights from the same Philox draws, unbiasedness of
the importance-weighted tally, and the trained network's gain over the
uniform sampler."""

import math

import numpy as np
import pytest

from oracle import mlp
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


def small_ct(window=1.5):
    return wl.ct_instrument(n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=32, window=window, spot=10e-6)


def norm_for(spec):
    src = spec.components[0]
    hw = 0.5 * src["target_w"]
    e_mid = 0.5 * (src["e_min"] + src["e_max"])
    e_half = 0.5 * (src["e_max"] - src["e_min"])
    return dict(half_u=hw, half_v=0.5 * src["target_h"], x_shift=[0, 0, e_mid, 0],
                x_scale=[1.0 / 10e-6, 1.0 / 10e-6, 1.0 / e_half, 1.0 / math.pi])


def params(seed=7, noise=0.05):
    rng = np.random.default_rng(seed)
    return (wl.proposal_init(seed) + rng.normal(0, noise, mlp.N_PARAMS)).astype(np.float32)


def test_forward_matches_oracle(env):
    mcx, torch = env
    th = params()
    p = mcx.Proposal(0.2, 0.1, 0.1, [0] * 4, [1] * 4, params=th)
    assert np.array_equal(p.get_params(), th)
    x = np.random.default_rng(1).normal(size=(3000, 4)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    out = torch.empty((3000, 40), dtype=torch.float32, device="cuda")
    p.forward(xd, out)
    ref, _ = mlp.forward(th.astype(np.float64), x.astype(np.float64), mirror_bf16=True)
    got = out.cpu().numpy()
    # Both sides round every layer's activations and weights to BF16; the
    # remaining difference is FP32 (tensor cores) against FP64 accumulation.
    # Where the two pre-activations straddle a BF16 rounding boundary the
    # next layer's operand differs by one BF16 ulp (2^-8 relative), which
    # moves an output by ~1e-3 of the outputs' rms (measured on GB300: at most
    # 1.3e-3 (|ref| + rms), 99.9 % below 1e-4).
    rms = float(np.sqrt((ref ** 2).mean()))
    np.testing.assert_allclose(got, ref, rtol=2e-3, atol=2e-3 * rms)
    assert np.quantile(np.abs(got - ref) / (np.abs(ref) + rms), 0.99) < 1e-4


@pytest.mark.parametrize("n", [4096, 1003])
def test_gradients_match_oracle(env, n):
    """n = 1003 leaves a ragged last row tile and a ragged last split of the
    weight-gradient reduction (rows not a multiple of the staged chunk)."""
    mcx, torch = env
    th = params(11, 0.1)
    p = mcx.Proposal(0.2, 0.1, 0.1, [0] * 4, [1] * 4, params=th)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(n, 4)).astype(np.float32)
    t = rng.uniform(-1, 1, size=(n, 2)).astype(np.float32)
    w = (rng.uniform(0, 2, size=n) * (rng.random(n) < 0.6)).astype(np.float32)
    loss, g = p.loss_grad(*(torch.tensor(a, device="cuda") for a in (x, t, w)))
    L, gref = mlp.loss_and_grad(th.astype(np.float64), x.astype(np.float64), t.astype(np.float64),
                                w.astype(np.float64), mirror_bf16=True)
    assert loss == pytest.approx(L, rel=1e-5)
    # per tensor in Frobenius norm: 5e-3 where BF16 activations enter (the
    # forward's one-ulp flips, measured <= 2.4e-3), 1e-4 for the head bias,
    # whose gradient sums the FP32 output gradient only (measured 5e-5)
    at = 0
    for i, shape in enumerate(mlp.SHAPES):
        k = int(np.prod(shape))
        a, b = g[at:at + k].astype(np.float64), gref[at:at + k]
        at += k
        bound = 1e-4 if i == len(mlp.SHAPES) - 1 else 5e-3
        assert np.linalg.norm(a - b) <= bound * np.linalg.norm(b) + 1e-9, (shape, np.linalg.norm(a - b) / np.linalg.norm(b))


def test_sampled_starts_match_oracle(env, orc):
    mcx, torch = env
    spec = small_ct()
    nf = norm_for(spec)
    th = params(5, 0.05)
    alpha = 0.25
    p = mcx.Proposal(alpha, nf["half_u"], nf["half_v"], nf["x_shift"], nf["x_scale"], params=th)
    inst = mcx.Instrument(spec, precision="mixed")
    n, b, seed = 20_000, 5_000, 13
    st = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    p.sample(inst, b, n, seed, st)
    g = st.view(6, n).cpu().numpy().astype(np.float64)
    # oracle: same source draws (mode 32), network in FP64 with BF16 operands,
    # then the selector and Box-Muller uniforms that follow them
    ost = orc.sample_starts(spec, b, n, seed).astype(np.float64)
    np.testing.assert_array_equal(g[:3], ost[:3])            # sx, sy, E
    x = np.stack([(ost[0] - nf["x_shift"][0]) * nf["x_scale"][0],
                  (ost[1] - nf["x_shift"][1]) * nf["x_scale"][1],
                  (ost[2] - nf["x_shift"][2]) * nf["x_scale"][2],
                  np.full(n, (0.0 - nf["x_shift"][3]) * nf["x_scale"][3])], axis=1)
    o, _ = mlp.forward(th.astype(np.float64), x.astype(np.float32).astype(np.float64), mirror_bf16=True)
    j0 = 2 + 3                                               # spot (2) + aim and energy (3)
    u = np.array([[orc.uniform32(b + i, 0, seed, j0 + k) for k in range(3)] for i in range(n)])
    t, factor, comp, unif = mlp.sample(o, alpha, u[:, 0], u[:, 1], u[:, 2])
    tu, tv = g[3] / nf["half_u"], g[4] / nf["half_v"]
    err = np.maximum(np.abs(tu - t[:, 0]), np.abs(tv - t[:, 1]))
    # the uniform branch is exact arithmetic on the same draws
    assert err[unif].max() < 1e-6
    # the Gaussian branch inherits the network outputs' difference (~1e-3 of
    # their rms, see the forward test) through mu + sigma z; the mixture
    # component is chosen by comparing a draw with cumulative weights, so a
    # different choice can only come from a draw within that difference of a
    # cumulative weight (a tie): every aim point further off than 5e-3 must be
    # such a tie
    logpi = mlp.head(o)[0]
    cum = np.cumsum(np.exp(logpi), axis=1)
    v = (u[:, 0] - alpha) / (1 - alpha)
    margin = np.abs(cum - v[:, None]).min(axis=1)
    far = err > 5e-3
    assert np.all(margin[far] < 5e-3), (err[far], margin[far])
    assert (err < 1e-4).mean() > 0.995 and (err < 1e-3).mean() > 0.9995
    kram = ((spec.components[0]["e0"] - ost[2]) / ost[2]) / (
        (160 * math.log(8.0) - 140.0) / 140.0)
    wref = factor * kram
    close = ~far
    ok = close & (wref > 0) & (g[5] > 0)
    # weights (1/4)/q at the aim point: the density carries the same output
    # difference (measured <= 1.6e-3 relative)
    np.testing.assert_allclose(g[5][ok], wref[ok], rtol=5e-3)
    # zero weight (aim point outside the window) on one side only where the
    # aim point lies within its difference of the window's edge
    edge = np.abs(1.0 - np.maximum(np.abs(t[:, 0]), np.abs(t[:, 1]))) <= err + 1e-7
    zero_differs = (g[5] == 0) != (wref == 0)
    assert not np.any(zero_differs & close & ~edge)


def _relvar(inst, n):
    N, sw, sw2 = inst.monitor(2)
    m = sw.sum() / n
    return m, (sw2.sum() / n - m * m) / n / (m * m)


def test_learned_sampler_is_unbiased_and_trained_net_beats_uniform(env):
    mcx, torch = env
    spec = small_ct()
    nf = norm_for(spec)
    n_hist = 1 << 20
    # histories from the plain sampler
    base = mcx.Instrument(spec, precision="mixed")
    st = torch.empty(6 * n_hist, dtype=torch.float32, device="cuda")
    det = torch.empty(n_hist, dtype=torch.float32, device="cuda")
    base.sample_starts(0, n_hist, 6, st)
    base.trace_starts(st, n_hist, 0, det)
    p = mcx.Proposal(0.1, nf["half_u"], nf["half_v"], nf["x_shift"], nf["x_scale"],
                     params=wl.proposal_init(0).astype(np.float32))
    l0 = p.train(st, det, n_hist, epochs=1, batch=8192, lr=3e-3)
    l1 = p.train(st, det, n_hist, epochs=4, batch=8192, lr=3e-3)
    assert l1 < l0
    n = 1 << 21
    plain = mcx.Instrument(spec, precision="mixed")
    plain.trace_range(0, n, 100)
    learned = mcx.Instrument(spec, precision="mixed")
    buf = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    p.sample(learned, 0, n, 100, buf)
    learned.trace_starts(buf, n, 0)
    mp, rvp = _relvar(plain, n)
    ml, rvl = _relvar(learned, n)
    # unbiased: the two estimates of the mean detected weight agree
    z = (ml - mp) / math.sqrt(rvp * mp * mp + rvl * ml * ml)
    assert abs(z) < 5, (mp, ml, z)
    # the trained proposal lowers the relative variance at equal ray count
    assert rvl < 0.8 * rvp, (rvl, rvp)


def test_attached_proposal_equals_sample_then_trace(env):
    """mcx_proposal_attach: a trace of an instrument with the proposal
    attached (sampled and traced in 2^23-ray chunks, here two and a ragged
    third) equals sampling the same rays into a buffer and tracing it; after
    detaching, the instrument traces its own source again."""
    mcx, torch = env
    spec = small_ct()
    nf = norm_for(spec)
    p = mcx.Proposal(0.3, nf["half_u"], nf["half_v"], nf["x_shift"], nf["x_scale"], params=params(3, 0.05))
    n, b, seed, angle = (1 << 24) + 12_345, 777, 21, 0.4
    a = mcx.Instrument(spec, precision="mixed")
    a.attach(p, angle)
    a.trace_range(b, b + n, seed)
    ref = mcx.Instrument(spec, precision="mixed")
    buf = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    p.sample(ref, b, n, seed, buf, angle=angle)
    ref.trace_starts(buf, n, b)
    for c in (2,):
        Na, swa, sw2a = a.monitor(c)
        Nr, swr, sw2r = ref.monitor(c)
        assert np.array_equal(Na, Nr) and int(Na.sum()) > 0
        np.testing.assert_allclose(swa, swr, rtol=1e-12, atol=0)
        np.testing.assert_allclose(sw2a, sw2r, rtol=1e-12, atol=0)
    ta, tr = a.tallies(), ref.tallies()
    assert ta["n_emit"] == tr["n_emit"] == n
    np.testing.assert_allclose(a.loss(), ta["lost"], rtol=0, atol=0)
    np.testing.assert_allclose(ta["lost"], tr["lost"], rtol=1e-6, atol=1e-6)
    # detached: the source's own sampler again
    a.attach(None)
    a.reset()
    a.trace_range(0, 50_000, 3)
    plain = mcx.Instrument(spec, precision="mixed")
    plain.trace_range(0, 50_000, 3)
    assert np.array_equal(a.monitor(2)[0], plain.monitor(2)[0])
    with pytest.raises(mcx.McxError):
        mcx.Instrument(spec, precision="fp64").attach(p)


def test_training_with_per_row_angles(env):
    """mcx_proposal_train_angles with every row at angle c trains the same
    network as mcx_proposal_train at angle c, up to the summation order of
    the gradient's atomic reductions (two runs of either differ as much), and
    with two angles in the rows it trains a clearly different one."""
    mcx, torch = env
    spec = small_ct()
    nf = norm_for(spec)
    n = 1 << 16
    base = mcx.Instrument(spec, precision="mixed")
    st = torch.empty(6 * n, dtype=torch.float32, device="cuda")
    det = torch.empty(n, dtype=torch.float32, device="cuda")
    base.sample_starts(0, n, 6, st)
    base.trace_starts(st, n, 0, det)

    def fresh():
        return mcx.Proposal(0.1, nf["half_u"], nf["half_v"], nf["x_shift"], nf["x_scale"],
                            params=wl.proposal_init(0).astype(np.float32))

    a, a2, b, c = fresh(), fresh(), fresh(), fresh()
    la = a.train(st, det, n, angle=0.7, epochs=2, batch=8192, lr=3e-3)
    a2.train(st, det, n, angle=0.7, epochs=2, batch=8192, lr=3e-3)
    lb = b.train(st, det, n, epochs=2, batch=8192, lr=3e-3,
                 angles=torch.full((n,), 0.7, dtype=torch.float32, device="cuda"))
    assert lb == pytest.approx(la, rel=1e-3)
    pa, pa2, pb = a.get_params(), a2.get_params(), b.get_params()
    init = wl.proposal_init(0).astype(np.float32)
    step = float(np.linalg.norm(pa - init))            # how far training moved the network
    assert step > 0
    # reruns differ only by the order of the gradient's atomic sums: a few
    # 1e-3 of the training's own step (both pairs measured alike)
    assert float(np.linalg.norm(pa - pa2)) < 1e-2 * step
    assert float(np.linalg.norm(pa - pb)) < 1e-2 * step
    mixed = torch.where(torch.arange(n, device="cuda") % 2 == 0, 0.7, 1.9).to(torch.float32)
    c.train(st, det, n, epochs=2, batch=8192, lr=3e-3, angles=mixed)
    assert float(np.linalg.norm(pa - c.get_params())) > 5e-2 * step


def test_batch_with_attached_proposals_equals_each_alone(env):
    """A batch holding instruments with the proposal attached (one spanning
    two 2^23-ray waves), an instrument with its own source and a slit
    instrument equals each instrument traced alone (the attached ones
    through mcx_trace_range with the proposal), in the generic and the
    family-compiled batch kernel; the allocation-free batch refuses
    attached instruments."""
    mcx, torch = env
    nf = norm_for(small_ct())
    p = mcx.Proposal(0.3, nf["half_u"], nf["half_v"], nf["x_shift"], nf["x_scale"], params=params(3, 0.05))
    specs = [wl.ct_instrument(angle=0.3, n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=32, window=1.5,
                              spot=10e-6, instr_id=1),
             wl.ct_instrument(angle=0.0, n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=32, window=1.5,
                              spot=10e-6, instr_id=2),
             wl.ct_instrument(angle=1.1, n=32, voxel=4 * MM, n_pix=32, pix=8 * MM, ne=32, window=1.5,
                              spot=10e-6, instr_id=3),
             wl.flat_slit_instrument(instr_id=4)]
    budgets = [(1 << 23) + 5_000, 1_000_000, 3_000_001, 500_000]
    angles = {0: 0.3, 2: 1.1}
    seed = 31
    alone = []
    for i, (sp, bud) in enumerate(zip(specs, budgets)):
        g = mcx.Instrument(sp, precision="mixed")
        if i in angles:
            g.attach(p, angles[i])
        g.trace_range(0, bud, seed)
        alone.append(g)
    for compiled in (False, True):
        insts = [mcx.Instrument(sp, precision="mixed") for sp in specs]
        for i, th in angles.items():
            insts[i].attach(p, th)
        b = mcx.Batch(insts, budgets, chunk_rays=1 << 18)
        if compiled:
            b.specialize()
        b.trace(seed)
        for i, (sp, g) in enumerate(zip(specs, insts)):
            for c, comp in enumerate(sp.components):
                if not comp["type"].startswith("mon_"):
                    continue
                Na, swa, sw2a = g.monitor(c)
                Nr, swr, sw2r = alone[i].monitor(c)
                assert np.array_equal(Na, Nr), (compiled, i, c)
                np.testing.assert_allclose(swa, swr, rtol=1e-12, atol=0)
                np.testing.assert_allclose(sw2a, sw2r, rtol=1e-12, atol=0)
            assert g.tallies()["n_emit"] == alone[i].tallies()["n_emit"] == budgets[i]
        b.close()
    with pytest.raises(mcx.McxError):
        mcx.batch_trace_static(insts, budgets, seed)
