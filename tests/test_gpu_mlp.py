"""The learned proposal: network kernels against the FP64 oracle, training,
the validity of Metropolis-Hastings with the learned q, and what it gains
over the random walk.

Tolerances: FP32 forward and gradients against FP64, relative 1e-5 in the
norm (per element 1e-4 relative with a small absolute floor); Adam against
the oracle's update after one step, 1e-6 relative.
"""
import math
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import ess, learned, synth

pytestmark = pytest.mark.gpu


def _net(api, d, H, seed):
    m = api.MLP(d, hidden=H, seed=seed)
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, m.num_params).astype(np.float32)
    m.set_params(torch.from_numpy(p).cuda())
    mean = rng.normal(0, 1, d).astype(np.float32)
    in_scale = rng.uniform(0.5, 2.0, d).astype(np.float32)
    scale = rng.uniform(0.2, 1.0, d).astype(np.float32)
    m.set_scaling(torch.from_numpy(mean).cuda(), torch.from_numpy(in_scale).cuda(), torch.from_numpy(scale).cuda(), 1.0)
    return m, p.astype(np.float64), mean.astype(np.float64), in_scale.astype(np.float64), scale.astype(np.float64)


def test_forward_and_gradient_match_oracle(cuda_lib):
    api = cuda_lib
    d, H, B = 37, 48, 20
    m, p, mean, in_scale, scale = _net(api, d, H, 3)
    rng = np.random.default_rng(4)
    th = rng.normal(0, 1, (B, d)).astype(np.float32)
    y = (th + rng.normal(0, 0.5, (B, d))).astype(np.float32)
    out = m.forward(torch.from_numpy(th).cuda()).cpu().numpy()
    ref = oracle.mlp_forward(p, d, H, mean, in_scale, th.astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-5
    loss, g = m.loss_grad(torch.from_numpy(th).cuda(), torch.from_numpy(y).cuda())
    oloss, og = oracle.mlp_loss_grad(p, d, H, mean, in_scale, scale, th.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - oloss) <= 1e-5 * abs(oloss)
    g = g.cpu().numpy()
    assert np.linalg.norm(g - og) / np.linalg.norm(og) < 1e-5
    np.testing.assert_allclose(g, og, rtol=1e-3, atol=1e-5 * np.abs(og).max())
    # one Adam step from zero moments
    m.adam_step(lr=1e-2)
    newp = m.get_params().cpu().numpy()
    pp, mm, vv = p.copy(), np.zeros_like(p), np.zeros_like(p)
    oracle.adam_step(pp, np.ascontiguousarray(g.astype(np.float64)), mm, vv, 1, lr=1e-2)
    np.testing.assert_allclose(newp, pp, rtol=1e-6, atol=1e-7)
    m.close()


def test_training_fits_a_drift(cuda_lib):
    api = cuda_lib
    d, n = 12, 20000
    rng = np.random.default_rng(5)
    X = rng.normal(0, 1, (n, d)).astype(np.float32)
    Y = (X - 0.5 * X + 0.1 * rng.normal(size=(n, d))).astype(np.float32)  # mean reversion
    m = api.MLP(d, hidden=64, seed=1)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    m.fit_scaling(Xd, Yd, lam=1.0)
    losses = m.train(Xd, Yd, 1500, batch=256, lr=3e-3, seed=2).cpu().numpy()
    assert losses[-100:].mean() < losses[:20].mean() - 5.0, (losses[:20].mean(), losses[-100:].mean())
    # the learned mean move is -0.5 x (in units of the displacement scale)
    out = m.forward(Xd[:512]).cpu().numpy()
    sc = (Y - X).std(0)
    pred = out[:, :d] * sc
    err = np.abs(pred - (-0.5 * X[:512])).mean()
    assert err < 0.1, err
    m.close()


def _prior_draws(K, n, rng, alpha_P=0.5):
    from tests.test_gpu_mcmc import _prior_draws as pd
    return pd(K, n, rng, alpha_P)


def test_learned_q_keeps_the_target(cuda_lib):
    """An asymmetric, state-dependent q (strong constant drift, scale varying
    with theta): with the q ratio the chains still target the prior."""
    api = cuda_lib
    from tests.test_gpu_mcmc import _make_sampler
    K, C = 4, 512
    rng = np.random.default_rng(88)
    draws = _prior_draws(K, C, rng)
    s, th0, step, obs, pr = _make_sampler(api, K, C, 88, T=0, step_scale=0.1, draws=draws)
    D = s.D
    m = api.MLP(D, hidden=32, seed=9)
    p = m.get_params().cpu().numpy()
    H = 32
    nW3 = 2 * D * H
    oW3 = H * D + H + H * H + H
    p[oW3:oW3 + nW3] *= 5.0                           # f depends on theta
    p[oW3 + nW3:oW3 + nW3 + D] = 0.1                  # drift in every coordinate (without the q ratio the chains would move off the prior)
    m.set_params(torch.from_numpy(p).cuda())
    sd = np.full(D, 0.1, np.float32)
    o = K * (K - 1) + (K - 1) + K
    sd[o:o + 2 * K] = 10.0
    m.set_scaling(torch.from_numpy(draws.mean(0)).cuda(), torch.from_numpy(draws.std(0) + 1e-3).cuda(),
                  torch.from_numpy(sd).cuda(), 1.0)
    s.set_proposal(m)
    s.step(150)
    th, lp, ll, na = s.state()
    acc = na.double().mean().item() / 150
    assert 0.05 < acc < 0.95, acc
    (pi, P, pt, mu, cov), _ = api.theta_to_params(th, K, pr)
    pt, mu = pt.cpu().numpy(), mu.cpu().numpy()
    n = C
    for k in range(K):
        mk = 0.1 if k < K // 2 else 0.9
        assert abs(pt[:, k].mean() - mk) < 0.012, (k, pt[:, k].mean())
    assert abs(mu[:, :, 0].mean() - 150) < 4 * 86.6 / math.sqrt(n * K) * 2
    assert abs(mu[:, :, 1].mean() - 75) < 4 * 43.3 / math.sqrt(n * K) * 2
    s.close()
    m.close()


def _timed(sampler, n):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lp, _ = sampler.step(n, trace_logpost=True)
    e1.record()
    torch.cuda.synchronize()
    return lp.cpu().numpy(), e0.elapsed_time(e1) / 1e3


def test_learned_proposal_vs_random_walk(cuda_lib):
    """Train on the random walk's history, then compare the effective sample
    size of the log posterior (Geyer ESS) over the same number of iterations,
    both started from the random walk's state after burn-in. The assertion is
    on ESS per iteration: at this toy size (K=4, T=3000) an iteration is a
    handful of launches and the network's two evaluations cost about half a
    random-walk iteration, while at the paper's sizes the likelihood is
    orders of magnitude dearer than the network (about 1 MFLOP per chain), so
    ESS per iteration is what carries over. ESS per second and the training
    time are printed."""
    api = cuda_lib
    from tests.test_gpu_mcmc import _theta_from_params
    K, C, T = 4, 128, 3000
    rng = np.random.default_rng(31)
    gen = synth.random_params(K, rng)
    obs = synth.sample_observations(gen, T, rng)
    D = api.theta_dim(K)
    base = _theta_from_params(K, gen.pi.astype(np.float64), gen.P.astype(np.float64),
                              gen.p_tremor.astype(np.float64), gen.mu.astype(np.float64),
                              gen.cov.astype(np.float64))
    th0 = torch.from_numpy((base[None] + 0.01 * rng.standard_normal((C, D))).astype(np.float32)).cuda()
    o = K * (K - 1) + (K - 1) + K
    step0 = np.full(D, 0.05, np.float32)
    step0[o:o + 2 * K] = 2.0                           # logits vs km-scale means
    xy, fl = torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda()
    pr = api.make_prior(K, alpha_P=0.5)

    def make(th, step, seed):
        return api.Sampler(K, th.contiguous(), torch.from_numpy(step).cuda(), seed, [0, T], xy, fl, prior=pr)

    # random-walk step multiplier tuned to an acceptance near 0.25
    best = None
    for mult in (0.25, 0.5, 1.0):
        s = make(th0, step0 * mult, 1)
        s.step(300)
        acc = learned.acceptance(s, 100)
        if best is None or abs(acc - 0.25) < abs(best[1] - 0.25):
            best = (mult, acc)
        s.close()
    step = step0 * best[0]
    rw = make(th0, step, 2)
    rw.step(6000)                                      # burn-in
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lp_rw, hist = rw.step(2000, trace_logpost=True, trace_theta=True)
    e1.record()
    torch.cuda.synchronize()
    t_rw = e0.elapsed_time(e1) / 1e3
    th_now, _, _, _ = rw.state()
    ls = make(th_now, step, 5)
    mlp, info = learned.fit_learned_proposal(ls, hist, lag=20, hidden=128, train_steps=2000, seed=3,
                                             lams=(0.8, 0.4, 0.2), target_accept=0.35, gamma=0.5)
    ls.step(200)
    lp_ml, t_ml = _timed(ls, 2000)
    lp_rw = lp_rw.cpu().numpy()
    e_rw, e_ml = ess.ess_chains(lp_rw), ess.ess_chains(lp_ml)
    gain_it = e_ml / e_rw
    gain_s = (e_ml / t_ml) / (e_rw / t_rw)
    print(f"RW x{best[0]} (acc {best[1]:.2f}): ESS {e_rw:.0f} in {t_rw:.3f}s ({e_rw / t_rw:.0f}/s); learned: ESS "
          f"{e_ml:.0f} in {t_ml:.3f}s ({e_ml / t_ml:.0f}/s); lam {info['lam']} gamma {info['gamma']}; pilot "
          f"{info['pilot']}; training {info['train_seconds']:.2f}s; gain per iteration {gain_it:.2f}x, "
          f"per second {gain_s:.2f}x")
    assert np.all(np.isfinite(lp_ml))
    assert info["losses"][-100:].mean() < info["losses"][:20].mean()
    assert gain_it > 1.1
    ls.close(); rw.close(); mlp.close()


def test_learned_sampler_full_size(cuda_lib):
    """The learned-proposal workload's launch: K=16 (d=351), T=2^20, 512
    chains, TF32 likelihood with FP32 recheck, a 2x256 network. A few random-
    walk iterations, a short training run on their trace, then learned
    iterations; the FP32 recheck of sampled chains' states matches the FP64
    oracle, the stored (TF32) log likelihood is within TF32's tolerance of
    it, and the stored log posterior is that plus the prior."""
    api = cuda_lib
    from paper_2003_03508_gb300 import chains
    K, T, C = 16, 1 << 20, 512
    prob = chains.tremor_problem(K, T, C, seed=9)
    pr = api.make_prior(K, alpha_P=0.5)
    step = torch.from_numpy(chains.base_steps(K) * 0.0625).cuda()
    s = api.Sampler(K, prob["theta0"], step, 9, [0, T], prob["xy"], prob["tremor"], prior=pr,
                    opts=api.make_opts(precision="tf32", recheck_fp32=1))
    _, hist = s.step(24, trace_theta=True)
    X, Y = learned.history_pairs(hist, lag=4)
    m = api.MLP(s.D, hidden=256, seed=2)
    m.fit_scaling(X, Y, lam=0.05)
    losses = m.train(X, Y, 50, batch=512, lr=1e-3, seed=3).cpu().numpy()
    assert np.all(np.isfinite(losses))
    m.set_lambda(0.05, 0.5)
    s.set_proposal(m)
    lp_tr, _ = s.step(3, trace_logpost=True)
    th, lp, ll, na = s.state()
    assert torch.all(torch.isfinite(lp_tr)) and torch.all(torch.isfinite(ll))
    (pi, P, p, mu, cov), lprior = api.theta_to_params(th, K, pr)
    assert torch.allclose(lp, ll + lprior, rtol=0, atol=1e-6 * float(ll.abs().max()))
    pick = [3, 411]
    prm = synth.HMMParams(*(t[pick].cpu().numpy() for t in (pi, P, p, mu, cov)))
    ref = oracle.loglik_batched(prm, prob["obs"].xy, prob["obs"].tremor, np.array([0, T], np.int64), n_threads=2)
    got = ll[pick].cpu().numpy()
    rep = s.fp32_report()[0][pick].cpu().numpy()
    print("K=16 T=2^20 512 chains: stored (TF32) log L rel err vs oracle", np.abs(got - ref) / np.abs(ref),
          "FP32 report", np.abs(rep - ref) / np.abs(ref))
    # the stored values are the sampler's TF32 ones; the recheck reports FP32
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref))
    assert np.all(np.abs(rep - ref) <= 1e-6 * np.abs(ref))
    s.close(); m.close()
