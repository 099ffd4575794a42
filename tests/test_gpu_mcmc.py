"""The random-walk Metropolis-Hastings layer (hmm_mcmc_step) against the oracle.

* theta -> parameters and log prior + log Jacobian: parity with the FP64
  oracle (the oracle itself is pinned against scipy and finite differences).
* Proposals are recomputed from the oracle's Philox draws and must match
  bit for bit; every accept/reject decision must equal the Metropolis-
  Hastings rule applied with the oracle's uniform (Section "Monte Carlo
  Markov Chains").
* With the likelihood switched off (T = 0: log L = 0) the chains target the
  prior: started at exact prior draws, they must keep the prior's moments.
  A wrong Jacobian or acceptance rule makes them drift.
* One call of n iterations (a CUDA graph replay) equals n calls of one.
* The FP32 recheck of accepted proposals is a separate report: it matches
  the oracle and never changes the values the acceptance rule compares.
* A checkpoint (hmm_sampler_save/load) resumes bit for bit, for the random
  walk, the t-walk and the learned proposal.
"""
import math

import numpy as np
import pytest
import torch
from scipy.stats import invwishart

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu


def _oprior(api_prior):
    return dict(alpha_P=api_prior.alpha_P, alpha_pi=api_prior.alpha_pi, p_mean_lo=api_prior.p_mean_lo,
                p_mean_hi=api_prior.p_mean_hi, p_var=api_prior.p_var, box=tuple(api_prior.box),
                iw_df=api_prior.iw_df)


def _theta_from_params(K, pi, P, p, mu, cov):
    th = []
    for i in range(K):
        th += [math.log(P[i, j] / P[i, i]) for j in range(K) if j != i]
    th += [math.log(pi[k] / pi[0]) for k in range(1, K)]
    th += [math.log(x / (1 - x)) for x in p]
    th += list(np.asarray(mu).reshape(-1))
    sx, sy = np.sqrt(cov[:, 0]), np.sqrt(cov[:, 2])
    for k in range(K):
        th += [math.log(sx[k]), math.log(sy[k])]
    th += [math.atanh(cov[k, 1] / (sx[k] * sy[k])) for k in range(K)]
    return np.array(th)


def _prior_draws(K, n, rng, alpha_P, alpha_pi=1.0):
    """Exact draws from the prior (host, numpy/scipy), as theta vectors."""
    out = []
    for _ in range(n):
        P = np.stack([rng.dirichlet(np.full(K, alpha_P)) for _ in range(K)])
        P = np.clip(P, 1e-30, None); P /= P.sum(1, keepdims=True)
        pi = rng.dirichlet(np.full(K, alpha_pi))
        p = np.empty(K)
        for k in range(K):
            m = 0.1 if k < K // 2 else 0.9
            a, b = m * m / 0.001, m / 0.001
            while True:
                x = rng.gamma(a, 1.0 / b)
                if 0 < x < 1:
                    break
            p[k] = x
        mu = np.column_stack([rng.uniform(0, 300, K), rng.uniform(0, 150, K)])
        cov = np.empty((K, 3))
        for k in range(K):
            S = invwishart.rvs(df=K, scale=np.eye(2), random_state=rng)
            cov[k] = (S[0, 0], S[0, 1], S[1, 1])
        out.append(_theta_from_params(K, pi, P, p, mu, cov))
    return np.array(out, dtype=np.float32)


@pytest.mark.parametrize("K", [3, 16, 32])
def test_theta_to_params_matches_oracle(cuda_lib, K):
    api = cuda_lib
    rng = np.random.default_rng(K)
    D = api.theta_dim(K)
    assert D == oracle.theta_dim(K)
    th = _prior_draws(K, 8, rng, alpha_P=0.5)
    pr = api.make_prior(K)
    (pi, P, p, mu, cov), lp = api.theta_to_params(torch.from_numpy(th).cuda(), K, pr)
    torch.cuda.synchronize()
    for c in range(th.shape[0]):
        (opi, oP, op, omu, ocov), olp = oracle.theta_to_params(th[c].astype(np.float64), K, _oprior(pr))
        np.testing.assert_allclose(pi[c].cpu().numpy(), opi, rtol=2e-7, atol=1e-30)
        np.testing.assert_allclose(P[c].cpu().numpy(), oP, rtol=2e-7, atol=1e-30)
        np.testing.assert_allclose(p[c].cpu().numpy(), op, rtol=2e-7)
        np.testing.assert_allclose(mu[c].cpu().numpy(), omu, rtol=2e-7)
        np.testing.assert_allclose(cov[c].cpu().numpy(), ocov, rtol=2e-6)
        assert abs(lp[c].item() - olp) <= 1e-9 * max(1.0, abs(olp)), (c, lp[c].item(), olp)


def _near_truth(K, C, gen, rng, scale=0.01):
    """Starting states near the generating parameters (for likelihood-on tests)."""
    base = _theta_from_params(K, gen.pi.astype(np.float64), gen.P.astype(np.float64),
                              gen.p_tremor.astype(np.float64), gen.mu.astype(np.float64),
                              gen.cov.astype(np.float64))
    return (base[None, :] + scale * rng.standard_normal((C, base.size))).astype(np.float32)


def _make_sampler(api, K, C, seed, T=0, step_scale=0.05, alpha_P=0.5, precision="fp32", recheck=0, draws=None):
    rng = np.random.default_rng(seed)
    D = api.theta_dim(K)
    if draws is not None:
        th0 = draws
    elif T > 0:
        th0 = None  # filled in below from the generating parameters
    else:
        th0 = _prior_draws(K, C, rng, alpha_P)
    step = np.full(D, step_scale, np.float32)
    o = K * (K - 1) + (K - 1) + K
    step[o:o + 2 * K] = 5.0 * step_scale * 20   # means move on the km scale
    gen = synth.random_params(K, rng)
    obs = synth.sample_observations(gen, T, rng)
    if th0 is None:
        th0 = _near_truth(K, C, gen, rng)
    pr = api.make_prior(K, alpha_P=alpha_P)
    s = api.Sampler(K, torch.from_numpy(th0).cuda(), torch.from_numpy(step).cuda(), seed, [0, T],
                    torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda(), prior=pr,
                    opts=api.make_opts(precision=precision, recheck_fp32=recheck))
    return s, th0, step, obs, pr


def test_proposals_and_decisions_match_oracle(cuda_lib):
    api = cuda_lib
    K, C, seed = 3, 16, 1234
    s, th0, step, obs, pr = _make_sampler(api, K, C, seed, T=0)
    D = s.D
    lp_trace, th_trace = s.step(3, trace_logpost=True, trace_theta=True)
    torch.cuda.synchronize()
    th_trace = th_trace.cpu().numpy()
    prior = _oprior(pr)
    cur = th0.copy()
    cur_lp = np.array([oracle.theta_to_params(cur[c].astype(np.float64), K, prior)[1] for c in range(C)])
    n_acc = 0
    for it in range(3):
        for c in range(C):
            z = np.array([oracle.normal(seed, 0, c, it, d) for d in range(D)])
            prop = (cur[c].astype(np.float64) + step.astype(np.float64) * z).astype(np.float32)
            plp = oracle.theta_to_params(prop.astype(np.float64), K, prior)[1]
            u = oracle.uniform(seed, 0, c, it, 0)
            # log L = log(sum pi) for T = 0 is zero up to float rounding of pi
            accept = math.isfinite(plp) and math.log(u) < plp - cur_lp[c]
            got = th_trace[it, c]
            if accept:
                assert np.array_equal(got, prop), (it, c)
                cur[c], cur_lp[c] = prop, plp
                n_acc += 1
            else:
                assert np.array_equal(got, cur[c]), (it, c)
        assert np.all(np.isfinite(lp_trace[it].cpu().numpy()))
    assert 0 < n_acc < 3 * C  # both outcomes occurred
    s.close()


def test_prior_is_invariant_without_likelihood(cuda_lib):
    api = cuda_lib
    K, C = 4, 512
    rng = np.random.default_rng(77)
    draws = _prior_draws(K, C, rng, alpha_P=0.5)
    s, th0, step, obs, pr = _make_sampler(api, K, C, 77, T=0, step_scale=0.15, draws=draws)
    s.step(150)
    th, lp, ll, na = s.state()
    torch.cuda.synchronize()
    acc = na.cpu().numpy().mean() / 150
    assert 0.1 < acc < 0.95, acc
    (pi, P, p, mu, cov), _ = api.theta_to_params(th, K, pr)
    p = p.cpu().numpy(); mu = mu.cpu().numpy(); pi = pi.cpu().numpy(); P = P.cpu().numpy()
    n = C
    # truncated Gamma(10, 100): mean 0.1, sd 0.0316; Gamma(810, 900): mean 0.9, sd 0.0316
    for k in range(K):
        m = 0.1 if k < K // 2 else 0.9
        assert abs(p[:, k].mean() - m) < 4 * 0.0316 / math.sqrt(n) * 3, (k, p[:, k].mean())
        assert abs(p[:, k].std() - 0.0316) < 0.006, (k, p[:, k].std())
    # uniform means: mean 150 / 75, sd 86.6 / 43.3
    assert abs(mu[:, :, 0].mean() - 150) < 4 * 86.6 / math.sqrt(n * K) * 2
    assert abs(mu[:, :, 1].mean() - 75) < 4 * 43.3 / math.sqrt(n * K) * 2
    assert abs(mu[:, :, 0].std() - 86.6) < 8 and abs(mu[:, :, 1].std() - 43.3) < 4
    # Dirichlet(1) on pi and Dirichlet(0.5) rows: every coordinate has mean 1/K
    assert np.all(np.abs(pi.mean(0) - 1 / K) < 0.04)
    assert np.all(np.abs(P.mean(0) - 1 / K) < 0.05)
    s.close()


def test_graph_replay_equals_single_steps(cuda_lib):
    api = cuda_lib
    K, C = 4, 32
    a, *_ = _make_sampler(api, K, C, 9, T=3000)
    b, *_ = _make_sampler(api, K, C, 9, T=3000)
    la, _ = a.step(12, trace_logpost=True)
    lb = torch.cat([b.step(1, trace_logpost=True)[0] for _ in range(12)])
    torch.cuda.synchronize()
    assert torch.equal(la, lb)
    ta, _, _, _ = a.state()
    tb, _, _, _ = b.state()
    assert torch.equal(ta, tb)
    assert a.launches_per_iter >= 5
    assert a.graph_active and not b.graph_active
    a.close(); b.close()


def test_stored_loglik_is_the_likelihood_of_the_state(cuda_lib):
    api = cuda_lib
    K, C = 6, 24
    s, th0, step, obs, pr = _make_sampler(api, K, C, 21, T=5000, step_scale=0.02)
    s.step(20)
    th, lp, ll, na = s.state()
    (pi, P, p, mu, cov), lprior = api.theta_to_params(th, K, pr)
    ctx = api.default_context()
    ref = ctx.hmm_loglik_batched(pi.contiguous(), P.contiguous(), p.contiguous(), mu.contiguous(),
                                 cov.contiguous(), [0, obs.T], torch.from_numpy(obs.xy).cuda(),
                                 torch.from_numpy(obs.tremor).cuda())
    torch.cuda.synchronize()
    assert torch.all(torch.isfinite(ll)) and na.sum().item() > 0
    assert torch.allclose(ll, ref, rtol=0, atol=0)
    assert torch.allclose(lp, ll + lprior, rtol=0, atol=1e-9)
    # the oracle agrees on a few chains
    for c in (0, 7, 23):
        prm = (pi[c].cpu().numpy(), P[c].cpu().numpy(), p[c].cpu().numpy(), mu[c].cpu().numpy(),
               cov[c].cpu().numpy())
        o = oracle.loglik(prm, obs.xy, obs.tremor)
        assert abs(ll[c].item() - o) <= 1e-6 * abs(o) + 1e-4
    s.close()


def test_fp32_recheck_reports_and_leaves_the_chains_alone(cuda_lib):
    """The FP32 recheck of the accepted proposals is a report: a TF32
    sampler with it on, stepped one iteration per call (a recheck after every
    call), moves exactly like the same sampler with it off stepped in one
    call, so no acceptance ratio ever mixes an FP32 value with a TF32 one.
    The stored log likelihoods stay the TF32 evaluations of the states; the
    report holds FP32 values that match the FP64 oracle."""
    api = cuda_lib
    K, C, n = 6, 24, 20
    a, th0, step, obs, pr = _make_sampler(api, K, C, 21, T=5000, step_scale=0.02, precision="tf32", recheck=1)
    b, *_ = _make_sampler(api, K, C, 21, T=5000, step_scale=0.02, precision="tf32", recheck=0)
    assert torch.isnan(a.fp32_report()[0]).all()  # nothing rechecked yet
    la = torch.cat([a.step(1, trace_logpost=True)[0] for _ in range(n)])
    lb, _ = b.step(n, trace_logpost=True)
    ta, lpa, lla, naa = a.state()
    tb, lpb, llb, nab = b.state()
    torch.cuda.synchronize()
    assert torch.equal(la, lb) and torch.equal(ta, tb) and torch.equal(lpa, lpb) and torch.equal(lla, llb)
    assert torch.equal(naa, nab) and naa.sum().item() > 0
    (pi, P, p, mu, cov), _ = api.theta_to_params(ta, K, pr)
    xy, fl = torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda()
    ctx = api.default_context()
    tf = ctx.hmm_loglik_batched(pi.contiguous(), P.contiguous(), p.contiguous(), mu.contiguous(),
                                cov.contiguous(), [0, obs.T], xy, fl, opts=api.make_opts(precision="tf32"))
    rep, dmax = a.fp32_report()
    torch.cuda.synchronize()
    assert torch.equal(lla, tf)  # the stored values are the sampler's own precision
    rep = rep.cpu().numpy()
    for c in range(C):
        prm = tuple(t[c].cpu().numpy() for t in (pi, P, p, mu, cov))
        o = oracle.loglik(prm, obs.xy, obs.tremor)
        assert abs(rep[c] - o) <= 1e-6 * abs(o) + 1e-4, (c, rep[c], o)
    assert abs(dmax.item() - np.abs(rep - lla.cpu().numpy()).max()) <= 1e-9
    # an explicit recheck evaluates again and agrees with the automatic one
    ll2, _ = a.recheck()
    torch.cuda.synchronize()
    assert np.array_equal(ll2.cpu().numpy(), rep)
    a.close(); b.close()


def test_tf32_decisions_use_tf32_values_on_both_sides(cuda_lib):
    """Every accept/reject decision of a TF32 sampler with the FP32 recheck
    on, across call boundaries, equals the Metropolis-Hastings rule replayed
    on the host from the oracle's Philox draws, the oracle's log prior and
    the TF32 log likelihoods of the current state and of the proposal (the
    same batched TF32 evaluation at the same chunk length)."""
    api = cuda_lib
    K, C, seed, n = 4, 32, 31, 6
    rng = np.random.default_rng(seed)
    D = api.theta_dim(K)
    gen = synth.random_params(K, rng)
    obs = synth.sample_observations(gen, 4000, rng)
    th0 = _near_truth(K, C, gen, rng, scale=0.02)
    step = np.full(D, 0.01, np.float32)
    o0 = K * (K - 1) + (K - 1) + K
    step[o0:o0 + 2 * K] = 0.5
    pr = api.make_prior(K, alpha_P=0.5)
    xy, fl = torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda()
    opts = api.make_opts(precision="tf32", chunk_len=256, recheck_fp32=1)
    s = api.Sampler(K, torch.from_numpy(th0).cuda(), torch.from_numpy(step).cuda(), seed, [0, obs.T], xy, fl,
                    prior=pr, opts=opts)
    traces = [s.step(1, trace_theta=True)[1] for _ in range(n)]
    torch.cuda.synchronize()
    ctx = api.Context()
    prior = _oprior(pr)

    def tf32_loglik(thetas):
        (pi, P, p, mu, cov), _ = api.theta_to_params(torch.from_numpy(thetas).cuda(), K, pr)
        out = ctx.hmm_loglik_batched(pi.contiguous(), P.contiguous(), p.contiguous(), mu.contiguous(),
                                     cov.contiguous(), [0, obs.T], xy, fl,
                                     opts=api.make_opts(precision="tf32", chunk_len=256))
        return out.cpu().numpy()

    cur = th0.copy()
    cur_ll = tf32_loglik(cur)
    cur_lp = np.array([oracle.theta_to_params(cur[c].astype(np.float64), K, prior)[1] for c in range(C)])
    n_acc = 0
    for it in range(n):
        props = np.empty_like(cur)
        for c in range(C):
            z = np.array([oracle.normal(seed, 0, c, it, d) for d in range(D)])
            props[c] = (cur[c].astype(np.float64) + step.astype(np.float64) * z).astype(np.float32)
        pll = tf32_loglik(props)
        got = traces[it][0].cpu().numpy()
        for c in range(C):
            plp = oracle.theta_to_params(props[c].astype(np.float64), K, prior)[1]
            u = oracle.uniform(seed, 0, c, it, 0)
            accept = math.isfinite(plp) and math.log(u) < (pll[c] + plp) - (cur_ll[c] + cur_lp[c])
            if accept:
                assert np.array_equal(got[c], props[c]), (it, c)
                cur[c], cur_ll[c], cur_lp[c] = props[c], pll[c], plp
                n_acc += 1
            else:
                assert np.array_equal(got[c], cur[c]), (it, c)
    assert 0 < n_acc < n * C
    ctx.close(); s.close()


def _run_pair(api, make, n1, n2, tmp_path, setup=None):
    """Sampler A runs n1 iterations, is saved, runs n2 more; sampler B (made
    the same way) loads the checkpoint and runs n2: both must end equal."""
    a = make()
    b = make()
    if setup:
        setup(a)
        setup(b)
    a.step(n1)
    path = tmp_path / "ckpt.bin"
    a.save(path)
    la, _ = a.step(n2, trace_logpost=True)
    b.load(path)
    lb, _ = b.step(n2, trace_logpost=True)
    sa, sb = a.state(), b.state()
    torch.cuda.synchronize()
    assert torch.equal(la, lb)
    for x, y in zip(sa, sb):
        assert torch.equal(x, y)
    return a, b, path


def test_checkpoint_resumes_bit_for_bit(cuda_lib, tmp_path):
    api = cuda_lib
    K, C = 4, 16
    make = lambda: _make_sampler(api, K, C, 11, T=3000, precision="tf32", recheck=1)[0]  # noqa: E731
    a, b, path = _run_pair(api, make, 5, 7, tmp_path)
    ra, rb = a.fp32_report(), b.fp32_report()
    torch.cuda.synchronize()
    assert torch.equal(ra[0], rb[0])
    # a sampler of another shape, or a file that is not a checkpoint, is refused
    other = _make_sampler(api, K, C + 1, 11, T=3000)[0]
    with pytest.raises(api.HMMError) as e:
        other.load(path)
    assert e.value.code == api.HMM_EINVAL
    bad = tmp_path / "junk.bin"
    bad.write_bytes(b"not a checkpoint" * 10)
    with pytest.raises(api.HMMError) as e:
        a.load(bad)
    assert e.value.code == api.HMM_EINVAL
    with pytest.raises(api.HMMError):
        a.load(tmp_path / "missing.bin")
    a.close(); b.close(); other.close()


def test_checkpoint_resumes_twalk_and_learned(cuda_lib, tmp_path):
    api = cuda_lib
    K, C = 4, 16

    def make():
        return _make_sampler(api, K, C, 12, T=2000)[0]

    def twalk(s):
        th = s.state()[0]
        g = torch.Generator(device="cuda").manual_seed(5)
        s.set_twalk((th + 0.01 * torch.randn(th.shape, device="cuda", generator=g)).contiguous())

    a, b, _ = _run_pair(api, make, 4, 6, tmp_path, setup=twalk)
    ta, tb = a.twalk_state(), b.twalk_state()
    assert torch.equal(ta[0], tb[0]) and torch.equal(ta[1], tb[1])
    a.close(); b.close()

    D = api.theta_dim(K)
    nets = []

    def learned(s):
        m = api.MLP(D, hidden=32, seed=len(nets))
        nets.append(m)
        X = s.state()[0].repeat(8, 1).contiguous()
        Y = (X + 0.01 * torch.randn_like(X)).contiguous()
        m.fit_scaling(X, Y, 0.5)
        if len(nets) == 1:
            m.train(X, Y, 20, batch=64, lr=1e-3, seed=3)
        m.set_lambda(0.5, 0.3)
        s.set_proposal(m)

    # B's network starts different (other seed, untrained): the load overwrites it
    a, b, _ = _run_pair(api, make, 3, 5, tmp_path, setup=learned)
    pa, pb = nets[0].get_params(), nets[1].get_params()
    torch.cuda.synchronize()
    assert torch.equal(pa, pb)
    a.close(); b.close()
