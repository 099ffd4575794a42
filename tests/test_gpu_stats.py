"""E-step statistics on the GPU (hmm_expected_stats) against the FP64
oracle, and what they are for: the Fisher-identity gradient and the EM
update.

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
from paper_2003_03508_gb300 import grad, synth

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


def test_gradient_and_em_from_gpu_stats(cuda_lib):
    rng = np.random.default_rng(1400)
    truth = synth.random_params(5, rng)
    obs = synth.sample_observations(truth, 20000, rng)
    prm = synth.perturb_params(truth, rng, scale=0.05)
    st, _ = _gpu(cuda_lib, prm, obs.xy, obs.tremor)
    ref, _ = oracle.expected_stats(prm, obs.xy, obs.tremor)
    g = grad.loglik_gradient(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov, st)
    gr = grad.loglik_gradient(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov, ref)
    for a, b in zip(g, gr):
        np.testing.assert_allclose(a, b, rtol=1e-3, atol=1e-3 * (np.abs(b).max() + 1e-12))
    # one EM step from the GPU statistics raises the likelihood
    before = oracle.loglik(prm, obs.xy, obs.tremor)
    after = oracle.loglik(synth.HMMParams(*grad.em_update(st)), obs.xy, obs.tremor)
    assert after > before


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
