"""Pins of the proposal oracle (oracle/mlp.py): analytic gradients against
central finite differences, mixture log-densities against scipy, the sampler
against the mixture's own cell probabilities, the unit mean of importance
factors, and bfloat16 rounding against torch."""

import math

import numpy as np
import pytest
from scipy import stats

from oracle import mlp
from paper_2410_08747_gb300 import workloads as wl


def test_param_count_and_init():
    th = wl.proposal_init(0)
    assert th.size == mlp.N_PARAMS == 38824
    assert np.isfinite(th).all()


@pytest.mark.parametrize("mirror", [False, True])
def test_gradient_finite_differences(mirror):
    rng = np.random.default_rng(1)
    th = wl.proposal_init(3) + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = rng.normal(size=(7, 4))
    t = rng.uniform(-1, 1, size=(7, 2))
    w = rng.uniform(0.1, 2.0, size=7)
    L, g = mlp.loss_and_grad(th, x, t, w)
    assert L == pytest.approx(mlp.loss(th, x, t, w), rel=1e-14)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 150, replace=False),
                          np.arange(mlp.N_PARAMS - 40, mlp.N_PARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[i] = h
        fd = (mlp.loss(th + e, x, t, w) - mlp.loss(th - e, x, t, w)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i
    if mirror:
        # with bf16-rounded operands the gradient is of the rounded model; it
        # stays close to the exact one
        L2, g2 = mlp.loss_and_grad(th, x, t, w, mirror_bf16=True)
        assert abs(L2 - L) < 2e-2 * max(1.0, abs(L))
        assert np.linalg.norm(g2 - g) < 5e-2 * np.linalg.norm(g)


def _head_only(b4):
    th = wl.proposal_init(0)
    ps = mlp.unflatten(th)
    ps[6][:] = 0.0
    ps[7][:] = b4
    return mlp.flatten(ps)


def test_single_component_log_density_is_normal():
    s = math.exp(-1.0)
    r = mlp.LS_C * math.atanh((math.log(s) - mlp.LS_M) / mlp.LS_C)
    b4 = np.zeros((8, 5))
    b4[:, 0] = -60.0
    b4[2] = [40.0, 0.2, -0.1, r, r]
    th = _head_only(b4.ravel())
    rng = np.random.default_rng(2)
    x = rng.normal(size=(50, 4))
    t = rng.uniform(-1, 1, size=(50, 2))
    o, _ = mlp.forward(th, x)
    lq, _ = mlp.log_gmm(o, t)
    ref = stats.norm.logpdf(t[:, 0], 0.2, s) + stats.norm.logpdf(t[:, 1], -0.1, s)
    np.testing.assert_allclose(lq, ref, rtol=1e-12, atol=1e-12)


def test_two_component_mixture_density():
    b4 = np.zeros((8, 5))
    b4[:, 0] = -80.0
    b4[0] = [math.log(0.3), -0.4, 0.1, 0.5, -0.3]
    b4[1] = [math.log(0.7), 0.3, -0.2, -0.7, 0.2]
    th = _head_only(b4.ravel())
    t = np.random.default_rng(3).uniform(-1, 1, size=(40, 2))
    o, _ = mlp.forward(th, np.zeros((40, 4)))
    lq, _ = mlp.log_gmm(o, t)
    ls = lambda r: mlp.LS_C * math.tanh(r / mlp.LS_C) + mlp.LS_M
    dens = 0.0
    for p, c in ((0.3, b4[0]), (0.7, b4[1])):
        dens = dens + p * stats.norm.pdf(t[:, 0], c[1], math.exp(ls(c[3]))) \
                        * stats.norm.pdf(t[:, 1], c[2], math.exp(ls(c[4])))
    np.testing.assert_allclose(lq, np.log(dens), rtol=1e-10)


def test_sampler_matches_cell_probabilities_and_unit_weights():
    b4 = np.zeros((8, 5))
    b4[:, 0] = -80.0
    b4[0] = [math.log(0.6), -0.3, 0.2, -0.5, -0.8]
    b4[1] = [math.log(0.4), 0.5, -0.4, -1.0, -0.2]
    th = _head_only(b4.ravel())
    n, alpha = 200_000, 0.2
    rng = np.random.default_rng(4)
    o, _ = mlp.forward(th, np.zeros((n, 4)))
    t, f, k, unif = mlp.sample(o, alpha, rng.random(n), rng.random(n), rng.random(n))
    # importance factors integrate the uniform density over the square: mean 1
    assert abs(f.mean() - 1.0) < 5 * f.std() / math.sqrt(n)
    # 8x8 cells: expected counts from the mixture's CDF (scipy)
    edges = np.linspace(-1, 1, 9)
    ls = lambda r: mlp.LS_C * math.tanh(r / mlp.LS_C) + mlp.LS_M
    P = np.full((8, 8), alpha / 64)
    for p, c in ((0.6, b4[0]), (0.4, b4[1])):
        cu = np.diff(stats.norm.cdf(edges, c[1], math.exp(ls(c[3]))))
        cv = np.diff(stats.norm.cdf(edges, c[2], math.exp(ls(c[4]))))
        P += (1 - alpha) * p * np.outer(cu, cv)
    H, _, _ = np.histogram2d(t[:, 0], t[:, 1], bins=[edges, edges])
    E = n * P
    chi2 = ((H - E) ** 2 / E).sum()
    assert chi2 < 63 + 5 * math.sqrt(2 * 63)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.concatenate([np.random.default_rng(5).normal(size=5000) * 10.0 ** np.arange(-20, 30, 0.01)[:5000],
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 1.01171875]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)
