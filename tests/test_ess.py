"""ESS estimator pins: an AR(1) process x_t = phi x_{t-1} + e_t has the
integrated autocorrelation time (1 + phi) / (1 - phi); iid draws have 1."""
import numpy as np

from paper_2003_03508_gb300 import ess


def _ar1(phi, n, rng):
    e = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = e[0] / np.sqrt(1 - phi ** 2)
    for t in range(1, n):
        x[t] = phi * x[t - 1] + e[t]
    return x


def test_iid_has_unit_iat():
    rng = np.random.default_rng(0)
    assert abs(ess.iat(rng.standard_normal(200_000)) - 1.0) < 0.05


def test_ar1_iat():
    rng = np.random.default_rng(1)
    for phi in (0.5, 0.9, 0.97):
        want = (1 + phi) / (1 - phi)
        got = np.mean([ess.iat(_ar1(phi, 100_000, rng)) for _ in range(3)])
        assert abs(got - want) / want < 0.1, (phi, got, want)


def test_ess_chains_sums():
    rng = np.random.default_rng(2)
    tr = rng.standard_normal((50_000, 4))
    assert abs(ess.ess_chains(tr) - 200_000) / 200_000 < 0.1


def test_esjd_of_a_known_walk():
    """Expected squared jump distance: a walk with unit steps in every one of
    D coordinates, scaled by 2, has ESJD = D / 4."""
    import torch
    from paper_2003_03508_gb300 import learned
    n, C, D = 50, 3, 7
    steps = torch.ones(n, C, D)
    steps[::2] *= -1.0
    th = torch.cumsum(steps, dim=0)
    assert abs(learned.esjd(th, torch.full((D,), 2.0)) - D / 4) < 1e-6
