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


def _iat_from_rho(rho: np.ndarray) -> np.ndarray:
    """Initial monotone sequence IAT for autocorrelations rho [n, m] (one
    column per chain): pair sums kept up to the first non-positive one, made
    non-increasing, tau = -1 + 2 sum."""
    n, m = rho.shape
    if n < 4:
        return np.full(m, np.inf)
    npair = n // 2
    g = rho[0:2 * npair:2] + rho[1:2 * npair:2]                  # [npair, m]
    positive = g > 0
    # keep the leading run of positive pair sums in every column
    keep = np.cumprod(positive, axis=0).astype(bool)
    g = np.where(keep, g, np.inf)
    g = np.minimum.accumulate(g, axis=0)
    g = np.where(keep, g, 0.0)
    tau = -1.0 + 2.0 * g.sum(axis=0)
    tau = np.where(keep[0], tau, 1.0)
    bad = ~np.isfinite(rho).all(axis=0) | (rho[0] == 0)
    tau = np.where(bad, np.inf, np.maximum(tau, 1.0))
    return tau


def _autocorr_cols(x: np.ndarray) -> np.ndarray:
    """Autocorrelations of every column of x [n, m] (FFT, biased estimator)."""
    import scipy.fft as sfft
    n = x.shape[0]
    x = x - x.mean(axis=0, keepdims=True)
    f = sfft.rfft(x, 2 * n, axis=0, workers=-1)
    ac = sfft.irfft(f * np.conj(f), axis=0, workers=-1)[:n] / n
    with np.errstate(invalid="ignore", divide="ignore"):
        return ac / ac[0:1]


def iat(x: np.ndarray) -> float:
    """Integrated autocorrelation time by the initial monotone sequence."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 1)
    if x.shape[0] < 4:
        return float("inf")
    rho = autocorr(x[:, 0]).reshape(-1, 1)
    return float(_iat_from_rho(rho)[0])


def ess(x: np.ndarray) -> float:
    """ESS of one chain's trace."""
    x = np.asarray(x, dtype=np.float64)
    return x.size / iat(x)


def ess_chains(traces: np.ndarray) -> float:
    """Total ESS of independent chains: traces [n_iter, n_chains], summed over chains."""
    traces = np.asarray(traces, dtype=np.float64)
    n = traces.shape[0]
    if n < 4:
        return 0.0
    rho = _autocorr_cols(traces)
    tau = _iat_from_rho(rho)
    return float(np.sum(n / tau))
