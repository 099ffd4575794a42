"""E-step statistics on the GPU (hmm_expected_stats) against the FP64
oracle, and the library calls built on them: the Fisher-identity gradient
(hmm_loglik_grad, checked against central differences of the likelihood
oracle) and the EM update (hmm_em_step).

Tolerance: every statistic within 1e-5 relative of the oracle's, with an
absolute floor of 1e-5 x the largest entry of that statistic (the
per-step posteriors carry ~1e-6 absolute FP32 error; their sums over T
steps average it). The gradient built from the GPU statistics agrees with
the one from the oracle's within 1e-3 relative (it subtracts nearly equal
moments).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import fisher
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    st, ll = ctx.hmm_expected_stats(*api.to_device(prm), torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                                    torch.from_numpy(np.ascontiguousarray(tremor)).cuda(),
                                    opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in st.items()}, float(ll.item())


def _close(st, ref):
    for name in ref:
        scale = np.abs(ref[name]).max() + 1e-30
        np.testing.assert_allclose(st[name], ref[name], rtol=1e-5, atol=1e-5 * scale, err_msg=name)


@pytest.mark.parametrize("K", [2, 3, 16, 25, 32, 64])
def test_stats_parity(cuda_lib, K):
    rng = np.random.default_rng(1200 + K)
    prm = synth.random_params(K, rng)
    obs = synth.sample_observations(prm, 5000 + 3, rng)
    ref, rll = oracle.expected_stats(prm, obs.xy, obs.tremor)
    for L in (64, 0):
        st, ll = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=L)
        _close(st, ref)
        assert abs(ll - rll) <= 1e-6 * abs(rll)


@pytest.mark.parametrize("T", [2, 3, 65, 130])
def test_stats_small_T(cuda_lib, T):
    rng = np.random.default_rng(1300 + T)
    prm = synth.random_params(4, rng)
    obs = synth.sample_observations(prm, T, rng)
    ref, _ = oracle.expected_stats(prm, obs.xy, obs.tremor)
    st, _ = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=64)
    _close(st, ref)


def _lib_grad(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    g, ll = ctx.hmm_loglik_grad(*api.to_device(prm), torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                                torch.from_numpy(np.ascontiguousarray(tremor)).cuda(), opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return tuple(a.cpu().numpy() for a in g), float(ll.item())


@pytest.mark.parametrize("init_mode", [0, 1])
def test_gradient_matches_finite_differences_of_the_oracle(cuda_lib, init_mode):
    """hmm_loglik_grad in every parameter against central differences of the
    FP64 likelihood oracle (float32 parameters, the step taken as the
    difference of the rounded perturbed values)."""
    rng = np.random.default_rng(71)
    prm = synth.random_params(3, rng, diag=(0.6, 0.9))
    obs = synth.sample_observations(prm, 400, rng)
    g, ll = _lib_grad(cuda_lib, prm, obs.xy, obs.tremor, init_mode=init_mode, chunk_len=64)
    assert abs(ll - oracle.loglik(prm, obs.xy, obs.tremor, init_mode)) <= 1e-6 * abs(ll)
    rel = {"pi": 3e-3, "P": 3e-3, "p_tremor": 2e-3, "mu": 1e-2, "cov": 1e-2}
    for name, gk in zip(("pi", "P", "p_tremor", "mu", "cov"), g):
        flat = getattr(prm, name).reshape(-1)
        for idx in range(flat.size):
            base = float(flat[idx])
            h = max(abs(base), 1e-3) * 1e-3
            up, dn = np.float32(base + h), np.float32(base - h)
            flat[idx] = up
            lu = oracle.loglik(prm, obs.xy, obs.tremor, init_mode)
            flat[idx] = dn
            ld = oracle.loglik(prm, obs.xy, obs.tremor, init_mode)
            flat[idx] = base
            fd = (lu - ld) / (float(up) - float(dn))
            an = gk.reshape(-1)[idx]
            assert abs(fd - an) <= rel[name] * max(abs(fd), 1.0), (name, idx, fd, an)


def test_gradient_and_em_step_match_the_oracle(cuda_lib):
    """K=5, T=20000 away from the generating parameters: the library's
    gradient against the Fisher identity applied to the oracle's statistics,
    its EM step against the oracle's M-step, and EM raising the likelihood."""
    api = cuda_lib
    rng = np.random.default_rng(1400)
    truth = synth.random_params(5, rng)
    obs = synth.sample_observations(truth, 20000, rng)
    prm = synth.perturb_params(truth, rng, scale=0.05)
    g, ll = _lib_grad(api, prm, obs.xy, obs.tremor)
    ref, rll = oracle.expected_stats(prm, obs.xy, obs.tremor)
    gr = fisher.loglik_gradient(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov, ref)
    for a, b in zip(g, gr):
        np.testing.assert_allclose(a, b, rtol=1e-3, atol=1e-3 * (np.abs(b).max() + 1e-12))
    ctx = api.default_context()
    new, ll2 = ctx.hmm_em_step(*api.to_device(prm), torch.from_numpy(obs.xy).cuda(),
                               torch.from_numpy(obs.tremor).cuda())
    new = tuple(t.cpu().numpy() for t in new)
    want = fisher.em_update(ref)
    for a, b in zip(new, want):
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-4 * (np.abs(b).max() + 1e-12))
    assert abs(float(ll2.item()) - rll) <= 1e-6 * abs(rll)
    before = oracle.loglik(prm, obs.xy, obs.tremor)
    after = oracle.loglik(synth.HMMParams(*new), obs.xy, obs.tremor)
    assert after > before


def test_em_iterations_fit_the_generating_parameters(cuda_lib):
    """Twenty EM iterations on the GPU from a perturbed start: the
    likelihood never falls (beyond FP32 rounding) and ends above the
    generating parameters' on the same data."""
    api = cuda_lib
    rng = np.random.default_rng(1500)
    truth = synth.random_params(4, rng)
    obs = synth.sample_observations(truth, 30000, rng)
    prm = synth.perturb_params(truth, rng, scale=0.1)
    ctx = api.default_context()
    xy, fl = torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda()
    cur = api.to_device(prm)
    prev = -np.inf
    for _ in range(20):
        cur, ll = ctx.hmm_em_step(*cur, xy, fl)
        v = float(ll.item())
        assert v >= prev - 1e-6 * abs(v), (prev, v)
        prev = v
    final = oracle.loglik(synth.HMMParams(*(t.cpu().numpy() for t in cur)), obs.xy, obs.tremor)
    assert final >= oracle.loglik(truth, obs.xy, obs.tremor)


def test_em_step_rejects_transition_first(cuda_lib):
    api = cuda_lib
    rng = np.random.default_rng(1600)
    prm = synth.random_params(3, rng)
    obs = synth.sample_observations(prm, 100, rng)
    with pytest.raises(api.HMMError) as e:
        api.default_context().hmm_em_step(*api.to_device(prm), torch.from_numpy(obs.xy).cuda(),
                                          torch.from_numpy(obs.tremor).cuda(), opts=api.make_opts(init_mode=1))
    assert e.value.code == api.HMM_EUNSUPPORTED


def test_stats_long_sequence(cuda_lib):
    """K=25, T=2^20 (the single-sequence workload)."""
    d = synth.config_inputs("k25_t2p20")
    ref, rll = oracle.expected_stats(d["params"], d["xy"], d["tremor"])
    st, ll = _gpu(cuda_lib, d["params"], d["xy"], d["tremor"])
    T = len(d["tremor"])
    assert abs(st["N"].sum() - (T - 1)) <= 1e-6 * T
    assert abs(st["Gs"].sum() - T) <= 1e-6 * T
    _close(st, ref)
    assert abs(ll - rll) <= 1e-6 * abs(rll)
