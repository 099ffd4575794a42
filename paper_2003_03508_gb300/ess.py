"""Effective sample size of MCMC traces (host-side statistics).

Section "Monte Carlo Markov Chains" assesses stationarity by trace plots and
"the number of effective independent samples". The estimator here is
Geyer's initial monotone sequence estimator (Geyer, "Practical Markov chain
Monte Carlo", Statistical Science 1992): with autocorrelations rho_k, the
sums of adjacent pairs Gamma_m = rho_{2m} + rho_{2m+1} are kept while
positive, forced to be non-increasing, and the integrated autocorrelation
time is tau = -1 + 2 sum_m Gamma_m; ESS = n / tau.
"""
from __future__ import annotations

import numpy as np


def autocorr(x: np.ndarray) -> np.ndarray:
    """Autocorrelation of a 1-D series at lags 0..n-1 (FFT, biased estimator)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    x = x - x.mean()
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[:n] / n
    if ac[0] <= 0:
        return np.zeros(n)
    return ac / ac[0]


def iat(x: np.ndarray) -> float:
    """Integrated autocorrelation time by the initial monotone sequence."""
    rho = autocorr(x)
    n = rho.size
    if n < 4 or not np.isfinite(rho).all() or rho[0] == 0:
        return float("inf")
    gam = []
    for m in range(n // 2):
        g = rho[2 * m] + rho[2 * m + 1]
        if g <= 0:
            break
        gam.append(g)
    if not gam:
        return 1.0
    gam = np.minimum.accumulate(np.array(gam))
    return max(1.0, -1.0 + 2.0 * gam.sum())


def ess(x: np.ndarray) -> float:
    """ESS of one chain's trace."""
    x = np.asarray(x, dtype=np.float64)
    return x.size / iat(x)


def ess_chains(traces: np.ndarray) -> float:
    """Total ESS of independent chains: traces [n_iter, n_chains], summed over chains."""
    traces = np.asarray(traces, dtype=np.float64)
    return float(sum(ess(traces[:, c]) for c in range(traces.shape[1])))
