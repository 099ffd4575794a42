"""Fisher-identity gradient of log L and the EM (Baum-Welch) update from the
hidden chain's expected sufficient statistics -- the oracle's statement of
that algebra (test infrastructure only), applied to statistics from
``oracle.expected_stats``.

Fisher identity: the gradient of the log likelihood equals the posterior
expectation of the gradient of the complete-data log likelihood,
    log p(s, o) = log v0[s_0] + sum_{t>=1} log P[s_{t-1}, s_t] + sum_t log e_{s_t}(o_t),
so with N (expected transitions), G0, and the gamma-weighted emission sums:
    d/dP_ij    = N_ij / P_ij
    d/dp_k     = Gr_k / p_k - (Gs_k - Gr_k) / (1 - p_k)
    d/dmu_k    = Sigma_k^-1 (S_k - Gr_k mu_k)
    d/dSigma_k = 1/2 Sigma_k^-1 (Q_k - Gr_k Sigma_k) Sigma_k^-1,
    Q_k = sum_t gamma_t(k) [tremor] (o_t - mu_k)(o_t - mu_k)^T,
and for pi (emit-first) d/dpi_k = G0_k / pi_k. P and pi are treated as free
entries (no simplex constraint); the covariance is parameterised by
(sxx, sxy, syy), sxy entering both off-diagonal entries.

The EM update maximises the expected complete-data log likelihood:
P_ij = N_ij / sum_j N_ij, pi = G0, p_k = Gr_k / Gs_k, mu_k = S_k / Gr_k,
Sigma_k = Q_k / Gr_k. Pinned in tests/test_oracle_stats.py (central finite
differences of the likelihood oracle, EM monotonicity).
"""
from __future__ import annotations

import numpy as np


def loglik_gradient(pi, P, p, mu, cov, st, init_mode: int = 0):
    """d log L / d (pi, P, p_tremor, mu, cov) as float64 arrays of the
    parameters' shapes, from the statistics dict `st` that
    oracle.expected_stats returns (N [K, K]; G0, Gs, Gr, Sx, Sy, Sxx,
    Sxy, Syy [K])."""
    pi, P, p, mu, cov = (np.asarray(a, dtype=np.float64) for a in (pi, P, p, mu, cov))
    K = pi.shape[0]
    N = st["N"]
    with np.errstate(divide="ignore", invalid="ignore"):
        dP = np.where(P > 0, N / P, 0.0)
        if init_mode == 1:
            v0 = pi @ P
            r = np.where(v0 > 0, st["G0"] / v0, 0.0)
            dpi = P @ r
            dP = dP + np.outer(pi, r)
        else:
            dpi = np.where(pi > 0, st["G0"] / pi, 0.0)
        dp = st["Gr"] / p - (st["Gs"] - st["Gr"]) / (1.0 - p)
    dmu = np.zeros((K, 2))
    dcov = np.zeros((K, 3))
    for k in range(K):
        S = np.array([[cov[k, 0], cov[k, 1]], [cov[k, 1], cov[k, 2]]])
        Lam = np.linalg.inv(S)
        m = mu[k]
        g = st["Gr"][k]
        s1 = np.array([st["Sx"][k], st["Sy"][k]])
        s2 = np.array([[st["Sxx"][k], st["Sxy"][k]], [st["Sxy"][k], st["Syy"][k]]])
        Q = s2 - np.outer(m, s1) - np.outer(s1, m) + g * np.outer(m, m)
        dmu[k] = Lam @ (s1 - g * m)
        dS = 0.5 * Lam @ (Q - g * S) @ Lam
        dcov[k] = (dS[0, 0], 2.0 * dS[0, 1], dS[1, 1])
    return dpi, dP, dp, dmu, dcov


def em_update(st):
    """One Baum-Welch M-step from the statistics: (pi, P, p_tremor, mu, cov)
    as float32 arrays (emit-first initial convention)."""
    N = st["N"]
    K = N.shape[0]
    P = N / N.sum(axis=1, keepdims=True)
    pi = st["G0"] / st["G0"].sum()
    g = st["Gr"]
    p = g / st["Gs"]
    mu = np.stack([st["Sx"] / g, st["Sy"] / g], axis=1)
    cov = np.empty((K, 3))
    cov[:, 0] = st["Sxx"] / g - mu[:, 0] ** 2
    cov[:, 1] = st["Sxy"] / g - mu[:, 0] * mu[:, 1]
    cov[:, 2] = st["Syy"] / g - mu[:, 1] ** 2
    return tuple(a.astype(np.float32) for a in (pi, P, p, mu, cov))
