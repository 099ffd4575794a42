"""Pins for the MCMC part of the oracle (random numbers, transforms, priors).

* Philox4x32-10 against the known-answer vectors published with the
  generator (Salmon et al. 2011, Random123 distribution).
* Uniforms and normals: moments of 2^16 draws.
* theta -> parameters: constraints hold, and an inverse map written here
  recovers theta.
* log prior + log Jacobian: equals scipy's densities (Dirichlet rows of P,
  Dirichlet pi, truncated Gamma p_k, inverse-Wishart Sigma_k, uniform mu)
  plus log|det J| of the transform computed by central finite differences,
  up to one constant that must not depend on theta (Section "Model priors",
  Appendix A, as read in the oracle's header).
"""
import math

import numpy as np
import pytest
from scipy.stats import dirichlet, gamma, invwishart

import oracle


def test_philox_known_answers():
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert list(oracle.philox4x32_10(ctr, key)) == want


def test_uniform_and_normal_moments():
    n = 1 << 14
    u = np.array([oracle.uniform(7, 0, 3, 5, i) for i in range(n)])
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003
    z = np.array([oracle.normal(7, 0, 3, 5, i) for i in range(n)])
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1) < 0.04
    assert abs(np.mean(z ** 3)) < 0.1 and abs(np.mean(z ** 4) - 3) < 0.2
    # pairs from one counter are uncorrelated (cos and sin branches)
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 0.05


def _inverse(K, pi, P, p, mu, cov):
    """params -> theta, written directly from the definitions."""
    th = []
    for i in range(K):
        for j in range(K):
            if j != i:
                th.append(math.log(P[i, j] / P[i, i]))
    for k in range(1, K):
        th.append(math.log(pi[k] / pi[0]))
    th += [math.log(x / (1 - x)) for x in p]
    th += list(mu.reshape(-1))
    sx = np.sqrt(cov[:, 0]); sy = np.sqrt(cov[:, 2])
    for k in range(K):
        th += [math.log(sx[k]), math.log(sy[k])]
    th += [math.atanh(cov[k, 1] / (sx[k] * sy[k])) for k in range(K)]
    return np.array(th)


def _random_theta(K, rng):
    d = oracle.theta_dim(K)
    assert d == K * K + 6 * K - 1
    th = rng.normal(0, 1.0, d)
    o = K * (K - 1) + (K - 1) + K
    th[o:o + 2 * K] = np.column_stack([rng.uniform(10, 290, K), rng.uniform(10, 140, K)]).reshape(-1)
    th[o + 2 * K:o + 4 * K] = rng.uniform(1.5, 3.0, 2 * K)   # log sigma
    th[o + 4 * K:] = rng.uniform(-0.6, 0.6, K)               # atanh rho
    return th


@pytest.mark.parametrize("K", [2, 3, 5])
def test_transform_constraints_and_roundtrip(K):
    rng = np.random.default_rng(K)
    prior = oracle.default_prior(K)
    for _ in range(5):
        th = _random_theta(K, rng)
        (pi, P, p, mu, cov), lp = oracle.theta_to_params(th, K, prior)
        assert np.allclose(P.sum(1), 1, atol=1e-14) and np.all(P > 0)
        assert abs(pi.sum() - 1) < 1e-14 and np.all(pi > 0)
        assert np.all((p > 0) & (p < 1))
        assert np.all(cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2 > 0)
        np.testing.assert_allclose(_inverse(K, pi, P, p, mu, cov), th, rtol=1e-10, atol=1e-10)
        assert math.isfinite(lp)


def _free_coords(K, theta, prior):
    """The coordinates the densities are written in: P_ij (j != i), pi_1..,
    p, mu, (sxx, sxy, syy)."""
    (pi, P, p, mu, cov), _ = oracle.theta_to_params(theta, K, prior)
    out = []
    for i in range(K):
        out += [P[i, j] for j in range(K) if j != i]
    out += list(pi[1:]) + list(p) + list(mu.reshape(-1))
    out += list(cov.reshape(-1))
    return np.array(out)


def _scipy_logprior(K, params, prior):
    pi, P, p, mu, cov = params
    lp = 0.0
    for i in range(K):
        lp += dirichlet.logpdf(P[i], np.full(K, prior["alpha_P"]))
    lp += dirichlet.logpdf(pi, np.full(K, prior["alpha_pi"]))
    for k in range(K):
        m = prior["p_mean_lo"] if k < K // 2 else prior["p_mean_hi"]
        a, b = m * m / prior["p_var"], m / prior["p_var"]
        lp += gamma.logpdf(p[k], a, scale=1.0 / b)
    for k in range(K):
        S = np.array([[cov[k, 0], cov[k, 1]], [cov[k, 1], cov[k, 2]]])
        lp += invwishart.logpdf(S, df=prior["iw_df"], scale=np.eye(2))
    return lp


@pytest.mark.parametrize("K", [2, 3])
def test_log_density_equals_scipy_plus_jacobian(K):
    rng = np.random.default_rng(100 + K)
    prior = oracle.default_prior(K)
    consts = []
    for _ in range(4):
        th = _random_theta(K, rng)
        params, lp = oracle.theta_to_params(th, K, prior)
        # numeric Jacobian of theta -> free coordinates (square)
        d = th.size
        J = np.zeros((d, d))
        h = 1e-6
        for c in range(d):
            e = np.zeros(d); e[c] = h
            J[:, c] = (_free_coords(K, th + e, prior) - _free_coords(K, th - e, prior)) / (2 * h)
        sign, logdet = np.linalg.slogdet(J)
        assert sign != 0
        consts.append(lp - _scipy_logprior(K, params, prior) - logdet)
    consts = np.array(consts)
    assert np.ptp(consts) < 1e-5, consts


def test_mean_outside_box_has_zero_prior():
    K = 3
    rng = np.random.default_rng(9)
    prior = oracle.default_prior(K)
    th = _random_theta(K, rng)
    o = K * (K - 1) + (K - 1) + K
    th[o] = 400.0  # x of state 0 beyond the 300 km box
    _, lp = oracle.theta_to_params(th, K, prior)
    assert lp == -math.inf


def test_box_edges():
    # each side of the box [0, 300] x [0, 150] km bounds its own coordinate only
    K = 3
    rng = np.random.default_rng(10)
    prior = oracle.default_prior(K)
    o = K * (K - 1) + (K - 1) + K
    for x, y, inside in ((299.0, 149.0, True), (1.0, 1.0, True), (200.0, 100.0, True),
                         (301.0, 75.0, False), (-1.0, 75.0, False), (150.0, 151.0, False),
                         (150.0, -1.0, False)):
        th = _random_theta(K, rng)
        th[o], th[o + 1] = x, y
        _, lp = oracle.theta_to_params(th, K, prior)
        assert math.isfinite(lp) == inside, (x, y, lp)
