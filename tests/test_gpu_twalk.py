"""The t-walk on the GPU (HMM_PROPOSAL_TWALK) against the t-walk oracle.

Without data (T = 0) the target is the prior of the transformed parameters,
which the oracle evaluates; every proposal (side, kernel, subset, draws)
and every decision is then reproduced from the same Philox counters. With
prior draws as the two starting points the chains must keep the prior, and
with data the stored log likelihood must be the likelihood of the state.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import chains, synth

pytestmark = pytest.mark.gpu


def _oprior(pr):
    return dict(alpha_P=pr.alpha_P, alpha_pi=pr.alpha_pi, p_mean_lo=pr.p_mean_lo, p_mean_hi=pr.p_mean_hi,
                p_var=pr.p_var, box=tuple(pr.box), iw_df=pr.iw_df)


def test_twalk_matches_oracle(cuda_lib):
    api = cuda_lib
    from tests.test_gpu_mcmc import _make_sampler, _prior_draws
    K, C, seed = 3, 16, 4321
    rng = np.random.default_rng(seed + 1)  # the sampler's first points come from default_rng(seed)
    s, th0, step, obs, pr = _make_sampler(api, K, C, seed, T=0)
    th2 = _prior_draws(K, C, rng, 0.5)
    s.set_twalk(torch.from_numpy(th2).cuda())
    prior = _oprior(pr)
    x, xp = th0.copy(), th2.copy()
    lx = np.array([oracle.theta_to_params(x[c].astype(np.float64), K, prior)[1] for c in range(C)])
    lxp = np.array([oracle.theta_to_params(xp[c].astype(np.float64), K, prior)[1] for c in range(C)])
    kinds, n_acc = [], 0
    for it in range(8):
        s.step(1)
        gx, _, _, _ = s.state()
        gxp, _ = s.twalk_state()
        gx, gxp = gx.cpu().numpy(), gxp.cpu().numpy()
        for c in range(C):
            side, kern, m, y, W = oracle.twalk_propose(x[c], xp[c], seed, c, it)
            kinds.append(kern)
            ly = oracle.theta_to_params(y.astype(np.float64), K, prior)[1]
            u = oracle.uniform(seed, 0, c, it, 0)
            cur = lx[c] if side == 0 else lxp[c]
            if W > -math.inf and math.isfinite(ly) and math.log(u) < ly - cur + W:
                n_acc += 1
                if side == 0:
                    x[c], lx[c] = y, ly
                else:
                    xp[c], lxp[c] = y, ly
            assert np.array_equal(gx[c], x[c]), (it, c, side, kern)
            assert np.array_equal(gxp[c], xp[c]), (it, c, side, kern)
    assert {"traverse", "walk"} <= set(kinds)
    assert 0 < n_acc < 8 * C
    s.close()


def test_twalk_keeps_the_prior(cuda_lib):
    api = cuda_lib
    from tests.test_gpu_mcmc import _make_sampler, _prior_draws
    K, C = 4, 512
    rng = np.random.default_rng(78)
    s, th0, step, obs, pr = _make_sampler(api, K, C, 78, T=0, draws=_prior_draws(K, C, rng, 0.5))
    s.set_twalk(torch.from_numpy(_prior_draws(K, C, rng, 0.5)).cuda())
    s.step(300)
    th, lp, ll, na = s.state()
    acc = na.double().mean().item() / 300
    assert 0.02 < acc < 0.95, acc
    (pi, P, p, mu, cov), _ = api.theta_to_params(th, K, pr)
    p, mu = p.cpu().numpy(), mu.cpu().numpy()
    n = C
    for k in range(K):
        m = 0.1 if k < K // 2 else 0.9
        assert abs(p[:, k].mean() - m) < 4 * 0.0316 / math.sqrt(n) * 3, (k, p[:, k].mean())
    assert abs(mu[:, :, 0].mean() - 150) < 4 * 86.6 / math.sqrt(n * K) * 2
    assert abs(mu[:, :, 1].mean() - 75) < 4 * 43.3 / math.sqrt(n * K) * 2
    assert abs(mu[:, :, 0].std() - 86.6) < 8 and abs(mu[:, :, 1].std() - 43.3) < 4
    s.close()


def test_twalk_with_data(cuda_lib):
    api = cuda_lib
    K, T, C = 4, 3000, 32
    prob = chains.tremor_problem(K, T, C, seed=23)
    pr = api.make_prior(K, alpha_P=0.5)
    s = api.Sampler(K, prob["theta0"], torch.from_numpy(chains.base_steps(K)).cuda(), 23, [0, T], prob["xy"],
                    prob["tremor"], prior=pr)
    th2 = prob["theta0"] + 0.02 * torch.randn_like(prob["theta0"])
    s.set_twalk(th2)
    lp_tr, _ = s.step(60, trace_logpost=True)
    th, lp, ll, na = s.state()
    assert torch.all(torch.isfinite(lp_tr)) and na.sum().item() > 0
    (pi, P, p, mu, cov), lprior = api.theta_to_params(th, K, pr)
    ctx = api.default_context()
    ref = ctx.hmm_loglik_batched(pi.contiguous(), P.contiguous(), p.contiguous(), mu.contiguous(),
                                 cov.contiguous(), [0, T], prob["xy"], prob["tremor"])
    torch.cuda.synchronize()
    assert torch.equal(ll, ref)
    assert torch.allclose(lp, ll + lprior, rtol=0, atol=1e-9)
    o = oracle.loglik(tuple(t[0].cpu().numpy() for t in (pi, P, p, mu, cov)), prob["obs"].xy, prob["obs"].tremor)
    assert abs(ll[0].item() - o) <= 1e-6 * abs(o)
    s.close()
