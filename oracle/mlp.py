"""FP64 oracle of the learned direction proposal (TEST INFRASTRUCTURE ONLY).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module; it never imports the GPU package.

The proposal is an importance-sampling density over the aim point (u, v) of
a source: q(u, v | x) with x = (source x, source y, energy, projection
angle).  The paper motivates it without defining it: most of an instrument's
rays are wasted (absorbed by a slit or missing the detector, Sec. 3.2) and an
energy-dispersive CT projection needs >= 1e7 rays (Sec. 5.1).  Here:

  network   x -> 3 hidden layers of 128 SiLU units -> 40 outputs
            (y = x W + b per layer, W stored [in, out])
  head      8 components k of a Gaussian mixture over the normalised aim point
            (u / hu, v / hv) in [-1, 1]^2: outputs (a, mu_u, mu_v, r_u, r_v)_k,
            pi = softmax(a), log sigma = C tanh(r / C) + M (C = 2.5, M = -2.5)
  loss      weighted negative log likelihood  -sum_i w_i log q(t_i | x_i) / sum_i w_i
  sampling  defensive mixture q_a = a U(square) + (1 - a) GMM; a sample outside
            the square gets weight 0; inside, the importance factor is
            (1/4) / q_a (the plain sampler is uniform on the square).

Everything is plain numpy in binary64; matrix products are library calls.
`bf16` (round to nearest even, as the GPU stores operands) can be applied to
the operands of layers 2-4 to mirror the tensor-core inputs.
"""

from __future__ import annotations

import numpy as np

HIDDEN = 128
N_COMP = 8
N_OUT = 5 * N_COMP
LS_C = 2.5
LS_M = -2.5
LOG_2PI = float(np.log(2.0 * np.pi))
SHAPES = [(4, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,),
          (HIDDEN, N_OUT), (N_OUT,)]
N_PARAMS = int(sum(np.prod(s) for s in SHAPES))


def unflatten(theta):
    """Flat parameter vector (W1, b1, W2, b2, W3, b3, W4, b4) -> list of arrays."""
    out, at = [], 0
    theta = np.asarray(theta, dtype=np.float64)
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[at:at + n].reshape(s))
        at += n
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def bf16(a):
    """Round binary64 values to bfloat16 (nearest, ties to even), as binary64."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, mirror_bf16=False):
    """Network outputs o [n, 40] and the cache for backward."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    q = bf16 if mirror_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1 + b1
    h1 = silu(z1)
    z2 = q(h1) @ q(W2) + b2
    h2 = silu(z2)
    z3 = q(h2) @ q(W3) + b3
    h3 = silu(z3)
    o = q(h3) @ q(W4) + b4
    return o, (x, z1, h1, z2, h2, z3, h3)


def head(o):
    """Mixture parameters from network outputs: log pi, mu_u, mu_v, log s_u, log s_v."""
    o = np.asarray(o, dtype=np.float64).reshape(-1, N_COMP, 5)
    a = o[:, :, 0]
    amax = a.max(axis=1, keepdims=True)
    logpi = a - (amax + np.log(np.exp(a - amax).sum(axis=1, keepdims=True)))
    lsu = LS_C * np.tanh(o[:, :, 3] / LS_C) + LS_M
    lsv = LS_C * np.tanh(o[:, :, 4] / LS_C) + LS_M
    return logpi, o[:, :, 1], o[:, :, 2], lsu, lsv


def log_gmm(o, t):
    """log q_gmm(t | o) per sample and the per-component terms."""
    logpi, mu, mv, lsu, lsv = head(o)
    t = np.asarray(t, dtype=np.float64)
    zu = (t[:, 0:1] - mu) / np.exp(lsu)
    zv = (t[:, 1:2] - mv) / np.exp(lsv)
    ell = logpi - 0.5 * zu * zu - lsu - 0.5 * zv * zv - lsv - LOG_2PI
    m = ell.max(axis=1, keepdims=True)
    lq = (m + np.log(np.exp(ell - m).sum(axis=1, keepdims=True)))[:, 0]
    return lq, (logpi, mu, mv, lsu, lsv, zu, zv, ell)


def loss(theta, x, t, w, mirror_bf16=False):
    o, _ = forward(theta, x, mirror_bf16)
    lq, _ = log_gmm(o, t)
    w = np.asarray(w, dtype=np.float64)
    return float(-(w * lq).sum() / w.sum())


def loss_and_grad(theta, x, t, w, mirror_bf16=False):
    """Weighted NLL and its gradient with respect to the flat parameters
    (analytic backward through the head, the SiLU layers and the products)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(theta)
    q = bf16 if mirror_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    o, (x, z1, h1, z2, h2, z3, h3) = forward(theta, x, mirror_bf16)
    lq, (logpi, mu, mv, lsu, lsv, zu, zv, ell) = log_gmm(o, t)
    w = np.asarray(w, dtype=np.float64)
    omega = w / w.sum()
    L = float(-(omega * lq).sum())
    # d log q / d head parameters; r = responsibilities
    r = np.exp(ell - lq[:, None])
    pi = np.exp(logpi)
    g_a = r - pi
    g_mu = r * zu / np.exp(lsu)
    g_mv = r * zv / np.exp(lsv)
    g_lsu = r * (zu * zu - 1.0)
    g_lsv = r * (zv * zv - 1.0)
    o3 = np.asarray(o).reshape(-1, N_COMP, 5)
    g_ru = g_lsu * (1.0 - np.tanh(o3[:, :, 3] / LS_C) ** 2)
    g_rv = g_lsv * (1.0 - np.tanh(o3[:, :, 4] / LS_C) ** 2)
    dO = -omega[:, None, None] * np.stack([g_a, g_mu, g_mv, g_ru, g_rv], axis=2)
    dO = dO.reshape(-1, N_OUT)
    # backward through the layers (operands as in the forward products)
    dW4 = q(h3).T @ dO
    db4 = dO.sum(axis=0)
    dz3 = (dO @ q(W4).T) * dsilu(z3)
    dW3 = q(h2).T @ dz3
    db3 = dz3.sum(axis=0)
    dz2 = (dz3 @ q(W3).T) * dsilu(z2)
    dW2 = q(h1).T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ q(W2).T) * dsilu(z1)
    dW1 = x.T @ dz1
    db1 = dz1.sum(axis=0)
    return L, flatten([dW1, db1, dW2, db2, dW3, db3, dW4, db4])


def q_alpha(o, t, alpha):
    """Defensive-mixture density in normalised aim coordinates."""
    lq, _ = log_gmm(o, t)
    t = np.asarray(t, dtype=np.float64)
    inside = (np.abs(t[:, 0]) <= 1.0) & (np.abs(t[:, 1]) <= 1.0)
    return alpha * 0.25 * inside + (1.0 - alpha) * np.exp(lq)


def sample(o, alpha, u_sel, u_a, u_b):
    """Aim points from the defensive mixture given uniforms, and their
    importance factor (1/4)/q_a (0 outside the square).  Component k is the
    first with cumulative pi > (u_sel - alpha)/(1 - alpha); its Gaussian is
    drawn by Box-Muller from (u_a, u_b)."""
    logpi, mu, mv, lsu, lsv = head(o)
    n = logpi.shape[0]
    u_sel, u_a, u_b = (np.asarray(v, dtype=np.float64) for v in (u_sel, u_a, u_b))
    t = np.zeros((n, 2))
    unif = u_sel < alpha
    t[unif, 0] = 2.0 * u_a[unif] - 1.0
    t[unif, 1] = 2.0 * u_b[unif] - 1.0
    g = ~unif
    c = np.cumsum(np.exp(logpi), axis=1)
    v = (u_sel - alpha) / (1.0 - alpha)
    k = np.minimum((c <= v[:, None]).sum(axis=1), N_COMP - 1)
    rad = np.sqrt(-2.0 * np.log(1.0 - u_a))
    z1 = rad * np.cos(2.0 * np.pi * u_b)
    z2 = rad * np.sin(2.0 * np.pi * u_b)
    idx = np.arange(n)
    t[g, 0] = mu[idx, k][g] + np.exp(lsu[idx, k][g]) * z1[g]
    t[g, 1] = mv[idx, k][g] + np.exp(lsv[idx, k][g]) * z2[g]
    qa = q_alpha(o, t, alpha)
    inside = (np.abs(t[:, 0]) <= 1.0) & (np.abs(t[:, 1]) <= 1.0)
    factor = np.where(inside, 0.25 / np.maximum(qa, 1e-300), 0.0)
    return t, factor, k, unif
