"""Pins for the E-step statistics oracle (oracle_expected_stats) and the
gradient / EM algebra built on them.

  * brute force over all K^T hidden paths (K = 3, T <= 6): the expected
    transition counts and gamma-weighted sums by enumeration;
  * totals: sum N = T - 1, sum Gs = T, sum Gr = number of tremor steps;
  * the Fisher-identity gradient equals central finite differences of the
    likelihood oracle in every parameter (pi, P, p, mu, Sigma), for both
    initial conventions -- an independent check of every statistic;
  * the EM update never lowers the likelihood (the EM monotonicity theorem).
"""
import itertools

import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle
from oracle import fisher
from paper_2003_03508_gb300 import synth


def _emis(prm, x, y, flag):
    out = np.empty(prm.K)
    for k in range(prm.K):
        pk = float(prm.p_tremor[k])
        if not flag:
            out[k] = 1.0 - pk
            continue
        c = prm.cov[k].astype(np.float64)
        out[k] = pk * multivariate_normal(mean=prm.mu[k].astype(np.float64),
                                          cov=[[c[0], c[1]], [c[1], c[2]]]).pdf([float(x), float(y)])
    return out


@pytest.mark.parametrize("T", [1, 2, 4, 6])
def test_bruteforce_stats(T):
    rng = np.random.default_rng(60 + T)
    prm = synth.random_params(3, rng, diag=(0.3, 0.8))
    obs = synth.sample_observations(prm, T, rng)
    st, _ = oracle.expected_stats(prm, obs.xy, obs.tremor)
    K = 3
    P = prm.P.astype(np.float64)
    E = np.array([_emis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t]) for t in range(T)])
    want = {k: np.zeros_like(v) for k, v in st.items()}
    Z = 0.0
    for path in itertools.product(range(K), repeat=T):
        w = float(prm.pi[path[0]]) * E[0, path[0]]
        for t in range(1, T):
            w *= P[path[t - 1], path[t]] * E[t, path[t]]
        Z += w
        want["G0"][path[0]] += w
        for t in range(T):
            k = path[t]
            want["Gs"][k] += w
            if obs.tremor[t]:
                x, y = float(obs.xy[t, 0]), float(obs.xy[t, 1])
                want["Gr"][k] += w
                want["Sx"][k] += w * x
                want["Sy"][k] += w * y
                want["Sxx"][k] += w * x * x
                want["Sxy"][k] += w * x * y
                want["Syy"][k] += w * y * y
            if t >= 1:
                want["N"][path[t - 1], k] += w
    for name in st:
        np.testing.assert_allclose(st[name], want[name] / Z, rtol=1e-9, atol=1e-9, err_msg=name)


def test_totals():
    d = synth.config_inputs("k4_t1e4")
    st, _ = oracle.expected_stats(d["params"], d["xy"], d["tremor"])
    T = len(d["tremor"])
    assert st["N"].sum() == pytest.approx(T - 1, rel=1e-10)
    assert st["Gs"].sum() == pytest.approx(T, rel=1e-10)
    assert st["Gr"].sum() == pytest.approx(int(np.sum(d["tremor"])), rel=1e-10)
    assert st["G0"].sum() == pytest.approx(1.0, rel=1e-12)


def _ll(prm, obs, mode):
    return oracle.loglik(prm, obs.xy, obs.tremor, mode)


@pytest.mark.parametrize("init_mode", [0, 1])
def test_gradient_matches_finite_differences(init_mode):
    rng = np.random.default_rng(71)
    prm = synth.random_params(3, rng, diag=(0.6, 0.9))
    obs = synth.sample_observations(prm, 400, rng)
    st, _ = oracle.expected_stats(prm, obs.xy, obs.tremor, init_mode)
    g = fisher.loglik_gradient(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov, st, init_mode)
    names = ("pi", "P", "p_tremor", "mu", "cov")
    rel = {"pi": 2e-3, "P": 2e-3, "p_tremor": 1e-3, "mu": 1e-2, "cov": 1e-2}
    for name, gk in zip(names, g):
        arr = getattr(prm, name)
        flat = arr.reshape(-1)
        for idx in range(flat.size):
            base = float(flat[idx])
            h = max(abs(base), 1e-3) * 1e-3
            up, dn = np.float32(base + h), np.float32(base - h)
            flat[idx] = up
            lu = _ll(prm, obs, init_mode)
            flat[idx] = dn
            ld = _ll(prm, obs, init_mode)
            flat[idx] = base
            fd = (lu - ld) / (float(up) - float(dn))
            an = gk.reshape(-1)[idx]
            assert abs(fd - an) <= rel[name] * max(abs(fd), 1.0), (name, idx, fd, an)


def test_em_update_does_not_lower_the_likelihood():
    rng = np.random.default_rng(5)
    truth = synth.random_params(4, rng)
    obs = synth.sample_observations(truth, 3000, rng)
    prm = synth.perturb_params(truth, rng) if hasattr(synth, "perturb_params") else truth
    prev = oracle.loglik(prm, obs.xy, obs.tremor)
    for _ in range(3):
        st, _ = oracle.expected_stats(prm, obs.xy, obs.tremor)
        new = synth.HMMParams(*fisher.em_update(st))
        cur = oracle.loglik(new, obs.xy, obs.tremor)
        assert cur >= prev - 1e-6 * abs(prev), (prev, cur)
        prm, prev = new, cur


MUTANTS = {
    "xi_wrong_time": ("z += fwd[(t - 1) * K + i] * (double)P[i * K + j] * w[j];",
                      "z += fwd[t * K + i] * (double)P[i * K + j] * w[j];"),
    "sxy_wrong": ("Sxy[k] += g * x * y;", "Sxy[k] += g * x * x;"),
    "gr_all_steps": ("                Gr[k] += g;\n", ""),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    import tempfile
    from pathlib import Path
    src = (Path(oracle.__file__).parent / "hmm_oracle.c").read_text()
    a, b = MUTANTS[name]
    assert a in src
    L = oracle.compile_variant(src.replace(a, b), tempfile.mkdtemp())
    rng = np.random.default_rng(72)
    prm = synth.random_params(3, rng, diag=(0.6, 0.9))
    obs = synth.sample_observations(prm, 200, rng)
    st, _ = oracle.expected_stats(prm, obs.xy, obs.tremor, 0, _L=L)
    g = fisher.loglik_gradient(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov, st, 0)
    # central differences from the unmodified likelihood oracle
    bad = False
    for name_, gk in zip(("P", "p_tremor", "mu", "cov"), g[1:]):
        flat = getattr(prm, name_).reshape(-1)
        for idx in range(flat.size):
            base = float(flat[idx])
            h = max(abs(base), 1e-3) * 1e-3
            up, dn = np.float32(base + h), np.float32(base - h)
            flat[idx] = up
            lu = _ll(prm, obs, 0)
            flat[idx] = dn
            ld = _ll(prm, obs, 0)
            flat[idx] = base
            fd = (lu - ld) / (float(up) - float(dn))
            bad = bad or abs(fd - gk.reshape(-1)[idx]) > 1e-2 * max(abs(fd), 1.0)
    assert bad, name
