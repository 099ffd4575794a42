"""The seeded input generator follows its stated recipe.

Every GPU parity case and the benchmark draw their inputs from
paper_2003_03508_gb300.synth, so its distributions are pinned here:
parameter ranges and constraints, the quiescent state, the hidden chain's
transition frequencies, tremor rates and location moments per state, the
uneven segment lengths, the sparse-tremor variant, and determinism under a
fixed seed.
"""
import numpy as np
import pytest

from paper_2003_03508_gb300 import synth


@pytest.mark.parametrize("K", [1, 2, 4, 25, 80])
def test_random_params_ranges(K):
    rng = np.random.default_rng(K)
    prm = synth.random_params(K, rng)
    assert prm.pi.dtype == np.float32 and prm.pi.shape == (K,)
    np.testing.assert_allclose(prm.pi, 1.0 / K, rtol=1e-6)
    P = prm.P.astype(np.float64)
    assert P.shape == (K, K) and np.all(P >= 0)
    np.testing.assert_allclose(P.sum(1), 1.0, atol=1e-6)
    if K > 1:
        d = np.diag(P)
        assert np.all((d >= 0.95 - 1e-6) & (d <= 0.995 + 1e-6))
    assert np.all((prm.p_tremor >= 0.05) & (prm.p_tremor <= 0.9))
    assert np.all((prm.mu[:, 0] >= 0) & (prm.mu[:, 0] <= 300) & (prm.mu[:, 1] >= 0) & (prm.mu[:, 1] <= 150))
    sx, sy = np.sqrt(prm.cov[:, 0].astype(np.float64)), np.sqrt(prm.cov[:, 2].astype(np.float64))
    assert np.all((sx >= 5 - 1e-4) & (sx <= 20 + 1e-4) & (sy >= 5 - 1e-4) & (sy <= 20 + 1e-4))
    rho = prm.cov[:, 1] / (sx * sy)
    assert np.all(np.abs(rho) <= 0.5 + 1e-5)


def test_offdiagonal_mass_is_spread_over_all_other_states():
    # Dirichlet(1) split: each off-diagonal share averages 1 / (K - 1)
    rng = np.random.default_rng(0)
    K = 5
    shares = []
    for _ in range(400):
        P = synth.random_params(K, rng).P.astype(np.float64)
        off = P[0, 1:] / (1 - P[0, 0])
        shares.append(off)
    m = np.mean(shares, axis=0)
    np.testing.assert_allclose(m, 1.0 / (K - 1), atol=0.03)


def test_quiescent_state():
    prm = synth.quiescent_params(25, np.random.default_rng(2))
    assert prm.p_tremor[24] == np.float32(0.001)
    assert tuple(prm.mu[24]) == (150.0, 75.0)
    assert tuple(prm.cov[24]) == (150.0 ** 2, 0.0, 150.0 ** 2)


def test_hidden_chain_transitions_and_emissions():
    rng = np.random.default_rng(5)
    K = 3
    prm = synth.random_params(K, rng, diag=(0.6, 0.8))
    T = 300_000
    obs = synth.sample_observations(prm, T, rng)
    s = obs.states
    assert obs.xy.shape == (T, 2) and obs.tremor.shape == (T,) and s.shape == (T,)
    # empirical transition frequencies against P
    counts = np.zeros((K, K))
    np.add.at(counts, (s[:-1], s[1:]), 1)
    freq = counts / counts.sum(1, keepdims=True)
    np.testing.assert_allclose(freq, prm.P, atol=0.01)
    for k in range(K):
        in_k = s == k
        # tremor rate per state
        assert abs(obs.tremor[in_k].mean() - prm.p_tremor[k]) < 0.01
        # location mean and covariance per state, tremor steps only
        xy = obs.xy[in_k & (obs.tremor == 1)].astype(np.float64)
        np.testing.assert_allclose(xy.mean(0), prm.mu[k], atol=0.5)
        C = np.cov(xy.T)
        want = np.array([[prm.cov[k, 0], prm.cov[k, 1]], [prm.cov[k, 1], prm.cov[k, 2]]])
        np.testing.assert_allclose(C, want, rtol=0.05, atol=2.0)
    # no-tremor steps carry no location
    assert np.all(obs.xy[obs.tremor == 0] == 0)


def test_first_state_follows_pi():
    prm = synth.random_params(3, np.random.default_rng(1))
    prm.pi[:] = np.float32([0.7, 0.2, 0.1])
    firsts = [synth.sample_observations(prm, 1, np.random.default_rng(i)).states[0] for i in range(3000)]
    np.testing.assert_allclose(np.bincount(firsts, minlength=3) / 3000, [0.7, 0.2, 0.1], atol=0.03)


def test_segments_uneven_and_summing_to_total():
    rng = np.random.default_rng(3)
    lens = synth.segment_lengths(64, 1 << 24, rng)
    assert lens.shape == (64,) and np.all(lens >= 1)
    assert abs(int(lens.sum()) - (1 << 24)) <= 64
    # log-uniform over three decades before rescaling: a wide spread of lengths
    assert lens.max() / lens.min() > 50
    prm = synth.random_params(4, rng)
    xy, fl, offs = synth.sample_segments(prm, [5, 0, 7], rng)
    assert list(offs) == [0, 5, 5, 12] and xy.shape == (12, 2) and fl.shape == (12,)


def test_batched_inputs_shapes_and_sparse_variant():
    d = synth.batched_inputs(K=8, T=5000, n_prop=6, seed=4, n_seg=3)
    assert d["params"].P.shape == (6, 8, 8) and d["params"].mu.shape == (6, 8, 2)
    assert d["offsets"][0] == 0 and d["offsets"][-1] == d["xy"].shape[0] == d["tremor"].shape[0]
    np.testing.assert_allclose(d["params"].P.sum(-1), 1.0, atol=1e-6)
    np.testing.assert_allclose(d["params"].pi.sum(-1), 1.0, atol=1e-6)
    sp = synth.batched_inputs(K=8, T=200_000, n_prop=2, seed=4, sparse=True)
    lo, hi = synth.SPARSE_P_RANGE
    assert np.all((sp["gen"].p_tremor >= lo) & (sp["gen"].p_tremor <= hi))
    assert sp["tremor"].mean() < hi


def test_seeded_determinism():
    a = synth.batched_inputs(K=4, T=3000, n_prop=3, seed=9, n_seg=2)
    b = synth.batched_inputs(K=4, T=3000, n_prop=3, seed=9, n_seg=2)
    for x, y in zip(a["params"].as_tuple(), b["params"].as_tuple()):
        assert np.array_equal(x, y)
    assert np.array_equal(a["xy"], b["xy"]) and np.array_equal(a["tremor"], b["tremor"])
    c = synth.batched_inputs(K=4, T=3000, n_prop=3, seed=10, n_seg=2)
    assert not np.array_equal(a["xy"], c["xy"])
