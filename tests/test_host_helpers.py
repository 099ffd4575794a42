"""Host-side helpers: the inverse parameter transform that starts the chains,
and the benchmark's count of no-tremor runs."""
import numpy as np

import bench
import oracle
from paper_2003_03508_gb300 import chains, synth


def test_theta_from_params_inverts_the_oracle_transform():
    for K, seed in ((2, 0), (4, 1), (7, 2)):
        prm = synth.random_params(K, np.random.default_rng(seed))
        prm.pi[:] = np.random.default_rng(seed + 10).dirichlet(np.ones(K)).astype(np.float32)
        th = chains.theta_from_params(K, *(a.astype(np.float64) for a in prm.as_tuple()))
        assert th.shape == (oracle.theta_dim(K),)
        (pi, P, p, mu, cov), lp = oracle.theta_to_params(th, K, oracle.default_prior(K))
        for got, want in ((pi, prm.pi), (P, prm.P), (p, prm.p_tremor), (mu, prm.mu), (cov, prm.cov)):
            np.testing.assert_allclose(got, want.astype(np.float64), rtol=1e-6, atol=1e-9)
        assert np.isfinite(lp)


def test_quiet_runs_counts_maximal_no_tremor_runs_among_chain_steps():
    # one segment: the first observation is not a chain step
    fl = np.array([0, 0, 0, 1, 0, 1, 1, 0, 0], np.uint8)
    assert sorted(bench._quiet_runs(fl, [0, 9]).tolist()) == [1, 2, 2]
    # two segments: runs do not cross the boundary, each segment drops its first step
    fl2 = np.array([1, 0, 0, 0, 0, 0, 1], np.uint8)
    assert sorted(bench._quiet_runs(fl2, [0, 3, 7]).tolist()) == [2, 2]
    assert bench._quiet_runs(np.ones(5, np.uint8), [0, 5]).size == 0
