"""Pins for the Viterbi oracle (oracle_viterbi) and the path score
(oracle_path_logjoint).

  * brute force over all K^T paths (K = 3, T <= 7, both initial
    conventions): the best score, and the best path where it is unique;
  * the path score recomputed from scipy's densities for a random path;
  * identical transition rows: every step chooses its own best state;
  * P = I: one state for the whole sequence, argmax of log pi + sum log e;
  * the returned score is the score of the returned path;
and planted mistakes are caught.
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


def _logemis(prm, x, y, flag):
    out = np.empty(prm.K)
    for k in range(prm.K):
        pk = float(prm.p_tremor[k])
        if not flag:
            out[k] = math.log1p(-pk)
            continue
        c = prm.cov[k].astype(np.float64)
        out[k] = math.log(pk) + multivariate_normal(mean=prm.mu[k].astype(np.float64),
                                                    cov=[[c[0], c[1]], [c[1], c[2]]]).logpdf([float(x), float(y)])
    return out


def _score(prm, obs, path, mode):
    P = prm.P.astype(np.float64)
    v0 = prm.pi.astype(np.float64) @ P if mode == 1 else prm.pi.astype(np.float64)
    s = math.log(v0[path[0]]) + _logemis(prm, obs.xy[0, 0], obs.xy[0, 1], obs.tremor[0])[path[0]]
    for t in range(1, len(path)):
        s += math.log(P[path[t - 1], path[t]]) + _logemis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t])[path[t]]
    return s


@pytest.mark.parametrize("T", [1, 2, 4, 7])
@pytest.mark.parametrize("mode", [0, 1])
def test_bruteforce(T, mode):
    rng = np.random.default_rng(80 + T)
    prm = synth.random_params(3, rng, diag=(0.3, 0.8))
    prm.pi[:] = np.float32([0.5, 0.3, 0.2])
    obs = synth.sample_observations(prm, T, rng)
    path, v = oracle.viterbi(prm, obs.xy, obs.tremor, mode)
    scores = {pa: _score(prm, obs, pa, mode) for pa in itertools.product(range(3), repeat=T)}
    best = max(scores.values())
    assert v == pytest.approx(best, rel=1e-12, abs=1e-12)
    winners = [pa for pa, s in scores.items() if s >= best - 1e-9 * abs(best)]
    if len(winners) == 1:
        assert tuple(path) == winners[0]


def test_path_score_matches_scipy():
    rng = np.random.default_rng(3)
    prm = synth.random_params(4, rng)
    obs = synth.sample_observations(prm, 50, rng)
    path = rng.integers(0, 4, 50).astype(np.int32)
    assert oracle.path_logjoint(prm, obs.xy, obs.tremor, path) == pytest.approx(_score(prm, obs, path, 0), rel=1e-12)


def test_identical_rows_choose_per_step():
    rng = np.random.default_rng(4)
    prm = synth.random_params(5, rng)
    w = rng.dirichlet(np.ones(5)).astype(np.float32)
    prm.P[:] = w[None, :]
    obs = synth.sample_observations(prm, 200, rng)
    path, _ = oracle.viterbi(prm, obs.xy, obs.tremor)
    for t in range(200):
        le = _logemis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t])
        base = np.log(prm.pi.astype(np.float64)) if t == 0 else np.log(w.astype(np.float64))
        assert path[t] == int(np.argmax(base + le))


def test_identity_transition_single_state():
    rng = np.random.default_rng(5)
    prm = synth.random_params(4, rng)
    prm.P[:] = np.eye(4, dtype=np.float32)
    obs = synth.sample_observations(prm, 60, rng)
    path, v = oracle.viterbi(prm, obs.xy, obs.tremor)
    tot = np.log(prm.pi.astype(np.float64))
    for t in range(60):
        tot += _logemis(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t])
    assert np.all(path == int(np.argmax(tot)))
    assert v == pytest.approx(tot.max(), rel=1e-12)


def test_returned_score_is_the_paths():
    d = synth.config_inputs("k4_t1e4")
    path, v = oracle.viterbi(d["params"], d["xy"], d["tremor"])
    assert v == pytest.approx(oracle.path_logjoint(d["params"], d["xy"], d["tremor"], path), rel=1e-12)
    assert v <= oracle.loglik(d["params"], d["xy"], d["tremor"])


MUTANTS = {
    "no_transition": ("double v = d[i] + log((double)P[i * K + j]);", "double v = d[i];"),
    "transposed": ("double v = d[i] + log((double)P[i * K + j]);", "double v = d[i] + log((double)P[j * K + i]);"),
    "no_first_emission": ("for (int k = 0; k < K; ++k) d[k] = log(d[k]) + le[k];",
                          "for (int k = 0; k < K; ++k) d[k] = log(d[k]);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    src = (Path(oracle.__file__).parent / "hmm_oracle.c").read_text()
    a, b = MUTANTS[name]
    assert a in src
    L = oracle.compile_variant(src.replace(a, b), tempfile.mkdtemp())
    caught = False
    for seed in range(86, 94):
        rng = np.random.default_rng(seed)
        prm = synth.random_params(3, rng, diag=(0.3, 0.8))
        obs = synth.sample_observations(prm, 6, rng)
        path, v = oracle.viterbi(prm, obs.xy, obs.tremor, 0, _L=L)
        best = max(_score(prm, obs, pa, 0) for pa in itertools.product(range(3), repeat=6))
        ok = v == pytest.approx(best, rel=1e-9) and _score(prm, obs, path, 0) == pytest.approx(best, rel=1e-9)
        caught = caught or not ok
    assert caught
