"""Pins for the posterior-state oracle (oracle_posterior, forward-backward).

gamma_t(k) = P(s_t = k | observations) is pinned by
  * brute force over all K^T hidden paths (K = 3, T <= 7, both initial
    conventions), with emissions from scipy's bivariate normal;
  * the closed form for identical transition rows P = 1 w^T (the hidden
    states are then independent: gamma_t ∝ w ∘ e(o_t) for t >= 2,
    ∝ pi ∘ e(o_1) at t = 1 under the emit-first convention);
  * the closed form for P = I (the state never changes: gamma_t is the
    same for every t, ∝ pi_k prod_t e_k(o_t));
  * rows summing to one and log L equal to the likelihood oracle's;
and planted mistakes in a copy of the oracle are caught.
"""
import itertools
import math
import tempfile
from pathlib import Path

import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle
from paper_2003_03508_gb300 import synth


def _emis(prm, x, y, flag):
    out = np.empty(prm.K)
    for k in range(prm.K):
        p = float(prm.p_tremor[k])
        if not flag:
            out[k] = 1.0 - p
            continue
        c = prm.cov[k].astype(np.float64)
        out[k] = p * multivariate_normal(mean=prm.mu[k].astype(np.float64),
                                         cov=[[c[0], c[1]], [c[1], c[2]]]).pdf([float(x), float(y)])
    return out


def _brute(prm, obs, init_mode):
    K, T = prm.K, len(obs.tremor)
    P = prm.P.astype(np.float64)
    pi = prm.pi.astype(np.float64)
    v0 = pi @ P if init_mode == 1 else pi
    E = np.array([_emis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t]) for t in range(T)])
    g = np.zeros((T, K))
    for path in itertools.product(range(K), repeat=T):
        w = v0[path[0]] * E[0, path[0]]
        for t in range(1, T):
            w *= P[path[t - 1], path[t]] * E[t, path[t]]
        for t in range(T):
            g[t, path[t]] += w
    return g / g.sum(axis=1, keepdims=True)


@pytest.mark.parametrize("T", [1, 2, 4, 7])
@pytest.mark.parametrize("init_mode", [0, 1])
def test_bruteforce(T, init_mode):
    rng = np.random.default_rng(40 + T)
    prm = synth.random_params(3, rng, diag=(0.3, 0.8))
    prm.pi[:] = np.float32([0.5, 0.3, 0.2])
    obs = synth.sample_observations(prm, T, rng)
    g, ll = oracle.posterior(prm, obs.xy, obs.tremor, init_mode)
    np.testing.assert_allclose(g, _brute(prm, obs, init_mode), rtol=1e-10, atol=1e-13)
    assert ll == pytest.approx(oracle.loglik(prm, obs.xy, obs.tremor, init_mode), rel=1e-13)


def test_identical_rows_independent_states():
    rng = np.random.default_rng(9)
    prm = synth.random_params(5, rng)
    w = rng.dirichlet(np.ones(5)).astype(np.float32)
    prm.P[:] = w[None, :]
    obs = synth.sample_observations(prm, 300, rng)
    g, _ = oracle.posterior(prm, obs.xy, obs.tremor)
    for t in (0, 1, 150, 299):
        e = _emis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t])
        want = (prm.pi.astype(np.float64) if t == 0 else w.astype(np.float64)) * e
        np.testing.assert_allclose(g[t], want / want.sum(), rtol=1e-9, atol=1e-12)


def test_identity_transition_constant_posterior():
    rng = np.random.default_rng(10)
    prm = synth.random_params(4, rng)
    prm.P[:] = np.eye(4, dtype=np.float32)
    obs = synth.sample_observations(prm, 40, rng)
    g, _ = oracle.posterior(prm, obs.xy, obs.tremor)
    logw = np.log(prm.pi.astype(np.float64))
    for t in range(40):
        logw = logw + np.log(_emis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t]))
    want = np.exp(logw - logw.max())
    want /= want.sum()
    for t in range(40):
        np.testing.assert_allclose(g[t], want, rtol=1e-8, atol=1e-12)


def test_rows_sum_to_one_long_sequence():
    d = synth.config_inputs("k4_t1e4")
    g, ll = oracle.posterior(d["params"], d["xy"], d["tremor"])
    assert np.all(np.abs(g.sum(axis=1) - 1) < 1e-12)
    assert ll == pytest.approx(oracle.loglik(d["params"], d["xy"], d["tremor"]), rel=1e-12)


MUTANTS = {
    "backward_transposed": ("v += (double)P[i * K + j] * exp(le[j] - m) * beta[j];",
                            "v += (double)P[j * K + i] * exp(le[j] - m) * beta[j];"),
    "backward_wrong_step": ("log_emissions(K, p, mu, cov, tremor[t], xy[2 * t], xy[2 * t + 1], le);\n        double m = max_of(K, le), n = 0.0;",
                            "log_emissions(K, p, mu, cov, tremor[t - 1], xy[2 * t - 2], xy[2 * t - 1], le);\n        double m = max_of(K, le), n = 0.0;"),
    "forward_only": ("gamma[t * K + k] = gamma[t * K + k] * beta[k] / s;", "gamma[t * K + k] = gamma[t * K + k];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = (Path(oracle.__file__).parent / "hmm_oracle.c").read_text()
    a, b = MUTANTS[name]
    assert a in src
    L = oracle.compile_variant(src.replace(a, b), tempfile.mkdtemp())
    rng = np.random.default_rng(44)
    prm = synth.random_params(3, rng, diag=(0.3, 0.8))
    obs = synth.sample_observations(prm, 5, rng)
    g, _ = oracle.posterior(prm, obs.xy, obs.tremor, 0, _L=L)
    assert not np.allclose(g, _brute(prm, obs, 0), rtol=1e-8, atol=1e-10)
