"""Seeded synthetic tremor-shaped inputs for the HMM likelihood.

This module only *samples* inputs. It contains no part of the likelihood
computation, so both the CUDA path's tests and the CPU oracle's tests can draw
their inputs from it.

What it samples follows the tremor HMM of Section 2 (the hidden-state model
behind Eq. "emission-matrix" and Eq. "likelihood func"):

* K hidden states; state k emits "no tremor" with probability 1 - p_k, or a
  tremor whose (x, y) location in km is bivariate normal N(mu_k, Sigma_k).
* A transition matrix P (the paper's Gamma) with rows summing to one, and an
  initial distribution pi (the paper's delta).

The Shikoku catalogue the paper fits (Section "Tremor dataset of the Shikoku
region": 105,000 hourly points) is not available, so these generators stand
in for it. Their shapes follow the workload recipe:

* P_ii ~ U(0.95, 0.995); the off-diagonal mass 1 - P_ii is split over the
  other K - 1 states by a Dirichlet(1) draw; pi is uniform.
* p_k ~ U(0.05, 0.9); mu_k ~ U([0, 300] x [0, 150]) km; sigma_x, sigma_y ~
  U(5, 20) km; correlation rho ~ U(-0.5, 0.5).  The covariance is passed as
  (sxx, sxy, syy) = (sigma_x^2, rho sigma_x sigma_y, sigma_y^2).
* Observations come from sampling the hidden chain: s_1 ~ pi, then
  s_{t+1} ~ P[s_t]; each step emits "no tremor" (flag 0, xy = 0) or a float32
  location (flag 1).

The hidden chain is sampled by holding times (a geometric stay in state i,
then a jump to j != i with probability proportional to P_ij), which is the same
Markov chain as step-by-step sampling but runs in O(number of jumps) Python
iterations.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "HMMParams",
    "Observations",
    "random_params",
    "quiescent_params",
    "sample_observations",
    "sample_segments",
    "perturb_params",
    "stack_params",
    "segment_lengths",
]


@dataclass
class HMMParams:
    """One parameter set, float32, in the layout the C ABI takes.

    pi: [K]; P: [K, K] row-major with P[i, j] = Pr(i -> j); p_tremor: [K];
    mu: [K, 2] (x, y) in km; cov: [K, 3] (sxx, sxy, syy) in km^2.
    """

    pi: np.ndarray
    P: np.ndarray
    p_tremor: np.ndarray
    mu: np.ndarray
    cov: np.ndarray

    @property
    def K(self) -> int:
        return int(self.pi.shape[0])

    def as_tuple(self):
        return (self.pi, self.P, self.p_tremor, self.mu, self.cov)


@dataclass
class Observations:
    """xy: [T, 2] float32 (km); tremor: [T] uint8, 1 = tremor at xy, 0 = none."""

    xy: np.ndarray
    tremor: np.ndarray
    states: np.ndarray = field(default=None, repr=False)

    @property
    def T(self) -> int:
        return int(self.tremor.shape[0])


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def random_params(K: int, rng: np.random.Generator, *, diag=(0.95, 0.995),
                  p_range=(0.05, 0.9), box=(300.0, 150.0), sigma=(5.0, 20.0),
                  rho=(-0.5, 0.5)) -> HMMParams:
    """Tremor-shaped random parameters (the recipe in the module docstring)."""
    P = np.zeros((K, K), dtype=np.float64)
    if K == 1:
        P[0, 0] = 1.0
    else:
        for i in range(K):
            d = rng.uniform(*diag)
            off = rng.dirichlet(np.ones(K - 1)) * (1.0 - d)
            P[i, :i] = off[:i]
            P[i, i] = d
            P[i, i + 1:] = off[i:]
    pi = np.full(K, 1.0 / K)
    p = rng.uniform(*p_range, size=K)
    mu = np.stack([rng.uniform(0, box[0], K), rng.uniform(0, box[1], K)], axis=1)
    sx = rng.uniform(*sigma, size=K)
    sy = rng.uniform(*sigma, size=K)
    r = rng.uniform(*rho, size=K)
    cov = np.stack([sx * sx, r * sx * sy, sy * sy], axis=1)
    return HMMParams(_f32(pi), _f32(P), _f32(p), _f32(mu), _f32(cov))


def quiescent_params(K: int, rng: np.random.Generator) -> HMMParams:
    """K-1 spatial states plus one quiescent state (p = 0.001, centred, broad).

    The quiescent state's location is not specified anywhere; it is read as
    mu = box centre (150, 75) km, sigma_x = sigma_y = 150 km, rho = 0.
    """
    prm = random_params(K, rng)
    prm.p_tremor[K - 1] = 0.001
    prm.mu[K - 1] = (150.0, 75.0)
    prm.cov[K - 1] = (150.0 ** 2, 0.0, 150.0 ** 2)
    return prm


def _sample_states(P: np.ndarray, pi: np.ndarray, T: int, rng: np.random.Generator) -> np.ndarray:
    K = P.shape[0]
    P64 = P.astype(np.float64)
    states = np.empty(T, dtype=np.int32)
    pi64 = pi.astype(np.float64)
    s = int(rng.choice(K, p=pi64 / pi64.sum()))
    t = 0
    while t < T:
        stay = float(P64[s, s])
        if stay >= 1.0 or K == 1:
            run = T - t
        else:
            # number of consecutive steps spent in s (>= 1), geometric
            run = int(rng.geometric(1.0 - stay))
        run = min(run, T - t)
        states[t:t + run] = s
        t += run
        if t >= T:
            break
        w = P64[s].copy()
        w[s] = 0.0
        tot = w.sum()
        if tot <= 0.0:
            states[t:] = s
            break
        s = int(rng.choice(K, p=w / tot))
    return states


def sample_observations(prm: HMMParams, T: int, rng: np.random.Generator) -> Observations:
    """Sample T observations from the HMM with parameters ``prm``."""
    T = int(T)
    if T == 0:
        return Observations(np.zeros((0, 2), np.float32), np.zeros(0, np.uint8),
                            np.zeros(0, np.int32))
    st = _sample_states(prm.P, prm.pi, T, rng)
    p = prm.p_tremor.astype(np.float64)[st]
    flag = (rng.random(T) < p).astype(np.uint8)
    z = rng.standard_normal((T, 2))
    cov = prm.cov.astype(np.float64)
    sxx, sxy, syy = cov[st, 0], cov[st, 1], cov[st, 2]
    # Cholesky factor of [[sxx, sxy], [sxy, syy]] for sampling only
    l11 = np.sqrt(sxx)
    l21 = sxy / l11
    l22 = np.sqrt(np.maximum(syy - l21 * l21, 0.0))
    mu = prm.mu.astype(np.float64)[st]
    x = mu[:, 0] + l11 * z[:, 0]
    y = mu[:, 1] + l21 * z[:, 0] + l22 * z[:, 1]
    xy = np.stack([x, y], axis=1).astype(np.float32)
    xy[flag == 0] = 0.0
    return Observations(np.ascontiguousarray(xy), flag, st)


def segment_lengths(n_seg: int, total: int, rng: np.random.Generator,
                    lo_exp: float = 3.0, hi_exp: float = 6.0) -> np.ndarray:
    """Uneven segment lengths, log-uniform in 10^lo..10^hi, rescaled to ~total."""
    raw = np.floor(10.0 ** rng.uniform(lo_exp, hi_exp, size=n_seg))
    scaled = np.maximum(1, np.floor(raw * (total / raw.sum()))).astype(np.int64)
    return scaled


def sample_segments(prm: HMMParams, lengths, rng: np.random.Generator):
    """Independent observation segments; returns (xy, tremor, offsets[n_seg+1])."""
    lengths = [int(n) for n in lengths]
    offs = np.zeros(len(lengths) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lengths)
    xy = np.zeros((int(offs[-1]), 2), dtype=np.float32)
    fl = np.zeros(int(offs[-1]), dtype=np.uint8)
    for s, n in enumerate(lengths):
        o = sample_observations(prm, n, rng)
        xy[offs[s]:offs[s + 1]] = o.xy
        fl[offs[s]:offs[s + 1]] = o.tremor
    return xy, fl, offs


def perturb_params(prm: HMMParams, rng: np.random.Generator, scale: float = 0.02) -> HMMParams:
    """A nearby parameter set, as an MCMC proposal would be (natural space).

    Transition rows are multiplied entry-wise by exp(scale * N(0, 1)) and
    renormalised; p_k, mu, sigma and rho move by small clipped amounts.
    """
    K = prm.K
    P = prm.P.astype(np.float64) * np.exp(scale * rng.standard_normal((K, K)))
    P /= P.sum(axis=1, keepdims=True)
    pi = prm.pi.astype(np.float64) * np.exp(scale * rng.standard_normal(K))
    pi /= pi.sum()
    p = np.clip(prm.p_tremor.astype(np.float64) + 0.5 * scale * rng.standard_normal(K), 1e-4, 1 - 1e-4)
    mu = prm.mu.astype(np.float64) + 25.0 * scale * rng.standard_normal((K, 2))
    cov = prm.cov.astype(np.float64)
    sx = np.sqrt(cov[:, 0]) * np.exp(scale * rng.standard_normal(K))
    sy = np.sqrt(cov[:, 2]) * np.exp(scale * rng.standard_normal(K))
    r = np.clip(cov[:, 1] / np.sqrt(cov[:, 0] * cov[:, 2]) + scale * rng.standard_normal(K), -0.95, 0.95)
    cov = np.stack([sx * sx, r * sx * sy, sy * sy], axis=1)
    return HMMParams(_f32(pi), _f32(P), _f32(p), _f32(mu), _f32(cov))


def stack_params(prms) -> HMMParams:
    """Stack proposals into [n_prop, ...] contiguous float32 arrays."""
    return HMMParams(*[_f32(np.stack([getattr(q, f) for q in prms]))
                       for f in ("pi", "P", "p_tremor", "mu", "cov")])


def config_inputs(name: str, seed: int | None = None):
    """Named workloads used by tests and the benchmark.

    Returns a dict with 'params' (HMMParams, stacked over proposals when
    batched), 'xy', 'tremor', 'offsets' (segment offsets, int64) and 'K'.
    """
    if name == "k4_t1e4":            # one parameter set, K=4, T=10^4
        rng = np.random.default_rng(1 if seed is None else seed)
        prm = random_params(4, rng)
        o = sample_observations(prm, 10_000, rng)
        return dict(K=4, params=prm, xy=o.xy, tremor=o.tremor,
                    offsets=np.array([0, o.T], np.int64))
    if name == "k25_t2p20":          # K=25 incl. one quiescent state, T=2^20
        rng = np.random.default_rng(2 if seed is None else seed)
        prm = quiescent_params(25, rng)
        o = sample_observations(prm, 1 << 20, rng)
        return dict(K=25, params=prm, xy=o.xy, tremor=o.tremor,
                    offsets=np.array([0, o.T], np.int64))
    raise KeyError(name)


SPARSE_P_RANGE = (0.002, 0.05)


def batched_inputs(K: int, T: int, n_prop: int, seed: int, n_seg: int = 1,
                   quiescent: bool = False, scale: float = 0.02, sparse: bool = False):
    """n_prop perturbed proposals around one generating parameter set.

    With n_seg > 1 the observations are n_seg independent segments of uneven
    (log-uniform) length summing to about T, shared by every proposal. With
    sparse=True every state's tremor probability is drawn from SPARSE_P_RANGE
    instead (hours with a tremor are rare; no-tremor runs average 20 to 500
    steps), the workload of the run-length shortcut.
    """
    rng = np.random.default_rng(seed)
    if sparse:
        gen = random_params(K, rng, p_range=SPARSE_P_RANGE)
    else:
        gen = quiescent_params(K, rng) if quiescent else random_params(K, rng)
    if n_seg == 1:
        o = sample_observations(gen, T, rng)
        xy, fl, offs = o.xy, o.tremor, np.array([0, T], np.int64)
    else:
        lens = segment_lengths(n_seg, T, rng)
        xy, fl, offs = sample_segments(gen, lens, rng)
    props = [perturb_params(gen, rng, scale) for _ in range(n_prop)]
    return dict(K=K, gen=gen, params=stack_params(props), xy=xy, tremor=fl, offsets=offs)
