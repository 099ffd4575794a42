"""Pins for the network oracle: its forward against a numpy composition of
the layers, its backpropagated gradient against central finite differences
of its own loss, and its Adam step (Kingma & Ba, ICLR 2015, Algorithm 1) against properties that
the algorithm's definition fixes without restating it: the first step from
zero moments, the closed form under a constant gradient, invariance to the
gradient's scale, and convergence to the minimiser of a quadratic."""
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


def _adam_run(p0, grads, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    p = np.array(p0, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    out = []
    for t, g in enumerate(grads, start=1):
        oracle.adam_step(p, np.ascontiguousarray(g, dtype=np.float64), m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        out.append(p.copy())
    return out


def test_adam_first_step_moves_lr_against_the_gradient_sign():
    """From zero moments the bias-corrected estimates are exactly g and g^2,
    so the first step is -lr g / (|g| + eps): -lr sign(g) for eps -> 0,
    whatever the gradient's magnitude."""
    rng = np.random.default_rng(3)
    g = rng.normal(size=64) * np.exp(rng.uniform(-8, 8, 64))
    p0 = rng.normal(size=64)
    (p1,) = _adam_run(p0, [g], lr=0.01, eps=0.0)
    np.testing.assert_allclose(p1 - p0, -0.01 * np.sign(g), rtol=1e-12, atol=0)
    (p1e,) = _adam_run(p0, [g], lr=0.01, eps=1e-3)
    np.testing.assert_allclose(p1e - p0, -0.01 * g / (np.abs(g) + 1e-3), rtol=1e-12, atol=0)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient the bias corrections make both moment
    estimates exact at every step (1 - beta^t cancels), so after t steps the
    parameters have moved by exactly t lr g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    g = rng.normal(size=32) * np.exp(rng.uniform(-5, 5, 32))
    p0 = rng.normal(size=32)
    traj = _adam_run(p0, [g] * 25, lr=3e-3, eps=1e-6)
    for t, p in enumerate(traj, start=1):
        np.testing.assert_allclose(p - p0, -t * 3e-3 * g / (np.abs(g) + 1e-6), rtol=1e-9, atol=1e-15)


def test_adam_is_invariant_to_gradient_scale():
    """eps = 0: m/sqrt(v) is homogeneous of degree 0 in the gradients, so
    multiplying every gradient by c > 0 leaves the iterates unchanged."""
    rng = np.random.default_rng(5)
    grads = [rng.normal(size=16) for _ in range(12)]
    p0 = rng.normal(size=16)
    a = _adam_run(p0, grads, eps=0.0)
    for c in (1e-4, 7.0, 1e5):
        b = _adam_run(p0, [c * g for g in grads], eps=0.0)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-14)


def test_adam_reaches_the_minimiser_of_a_separable_quadratic():
    """f(p) = sum a_i (p_i - c_i)^2 / 2 has its minimum at c; Adam with a
    decaying step (lr_t = lr / sqrt(t)) ends within a small fraction of the
    starting distance of it in every coordinate, despite curvatures that
    differ by 10^4."""
    rng = np.random.default_rng(6)
    n = 20
    a = np.exp(rng.uniform(-4.6, 4.6, n))
    c = rng.normal(0, 3, n)
    p = rng.normal(0, 3, n)
    start = np.abs(p - c).max()
    m = np.zeros(n)
    v = np.zeros(n)
    for t in range(1, 4001):
        g = a * (p - c)
        oracle.adam_step(p, np.ascontiguousarray(g), m, v, t, lr=0.3 / np.sqrt(t))
    assert np.abs(p - c).max() < 0.01 * start, np.abs(p - c).max()
