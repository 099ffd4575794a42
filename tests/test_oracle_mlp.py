"""Pins for the network oracle: its forward against a numpy composition of
the layers, its backpropagated gradient against central finite differences
of its own loss, and its Adam step against the update rule of Kingma & Ba
(ICLR 2015, Algorithm 1) written out here."""
import numpy as np

import oracle


def _setup(d=5, H=7, B=4, seed=0):
    rng = np.random.default_rng(seed)
    n = oracle.mlp_num_params(d, H)
    params = rng.normal(0, 0.4, n)
    mean = rng.normal(0, 1, d)
    in_scale = rng.uniform(0.5, 2.0, d)
    scale = rng.uniform(0.2, 1.0, d)
    theta = rng.normal(0, 1, (B, d))
    y = theta + rng.normal(0, 0.3, (B, d))
    return d, H, params, mean, in_scale, scale, theta, y


def _split(params, d, H):
    o = 0
    def take(n, shape):
        nonlocal o
        a = params[o:o + n].reshape(shape); o += n
        return a
    W1 = take(H * d, (H, d)); b1 = take(H, (H,)); W2 = take(H * H, (H, H)); b2 = take(H, (H,))
    W3 = take(2 * d * H, (2 * d, H)); b3 = take(2 * d, (2 * d,))
    return W1, b1, W2, b2, W3, b3


def test_forward_matches_numpy():
    d, H, params, mean, in_scale, scale, theta, y = _setup()
    W1, b1, W2, b2, W3, b3 = _split(params, d, H)
    x = (theta - mean) / in_scale
    ref = np.maximum(np.maximum(x @ W1.T + b1, 0) @ W2.T + b2, 0) @ W3.T + b3
    np.testing.assert_allclose(oracle.mlp_forward(params, d, H, mean, in_scale, theta), ref, rtol=1e-12, atol=1e-12)


def test_gradient_matches_finite_differences():
    d, H, params, mean, in_scale, scale, theta, y = _setup(seed=1)
    loss, g = oracle.mlp_loss_grad(params, d, H, mean, in_scale, scale, theta, y)
    h = 1e-6
    num = np.zeros_like(params)
    for i in range(params.size):
        e = np.zeros_like(params); e[i] = h
        num[i] = (oracle.mlp_loss_grad(params + e, d, H, mean, in_scale, scale, theta, y)[0] -
                  oracle.mlp_loss_grad(params - e, d, H, mean, in_scale, scale, theta, y)[0]) / (2 * h)
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7)


def test_loss_is_negative_log_density_without_constants():
    d, H, params, mean, in_scale, scale, theta, y = _setup(seed=2)
    out = oracle.mlp_forward(params, d, H, mean, in_scale, theta)
    fmu, fs = out[:, :d], np.clip(out[:, d:], -6, 3)
    sd = scale * np.exp(fs)
    # -log N(y; theta + scale f_mu, sd^2) = r^2/2 + log sd + log sqrt(2 pi), r in sd units
    nll = 0.5 * ((y - theta - scale * fmu) / sd) ** 2 + np.log(sd) + 0.5 * np.log(2 * np.pi)
    const = (np.log(scale).sum() + 0.5 * d * np.log(2 * np.pi))
    loss, _ = oracle.mlp_loss_grad(params, d, H, mean, in_scale, scale, theta, y)
    assert abs(loss - (nll.sum(1).mean() - const)) < 1e-10


def test_adam_step_rule():
    rng = np.random.default_rng(3)
    n = 50
    p = rng.normal(size=n); g = rng.normal(size=n); m = np.zeros(n); v = np.zeros(n)
    p0 = p.copy()
    for t in (1, 2, 3):
        gm = g * t
        mm = 0.9 * m + 0.1 * gm; vv = 0.999 * v + 0.001 * gm * gm
        want = p - 1e-2 * (mm / (1 - 0.9 ** t)) / (np.sqrt(vv / (1 - 0.999 ** t)) + 1e-8)
        oracle.adam_step(p, np.ascontiguousarray(gm), m, v, t, lr=1e-2)
        np.testing.assert_allclose(p, want, rtol=1e-14, atol=1e-14)
    assert not np.allclose(p, p0)
