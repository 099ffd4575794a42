"""Pins for the t-walk oracle (oracle/twalk_oracle.c) from the definitions of
its kernels, and runs on a Gaussian target.

The t-walk (Christen & Fox 2010) moves one of two points, on a random
subset of coordinates, by one of four kernels. Each pin recovers a kernel's
random variable from the proposals and tests it against its defining
distribution, or recomputes the Hastings factor from scipy's normal density:
  * subset sizes: Binomial(n, min(n, 4)/n) conditioned on >= 1;
  * traverse: beta = (y - r)/(r - h) follows g(beta) (CDF below), and the
    factor is (n_phi - 2) log beta;
  * walk: z = (y - h)/(h - r) follows the density prop. to 1/sqrt(1 + z)
    on [-a/(1+a), a], a = 1.5, and the factor is 0;
  * blow / hop: (y - r)/sigma and 3 (y - h)/sigma are standard normal, and
    the factor is the log ratio of the reverse and forward Gaussian
    proposal densities;
  * whole runs on N(0, I): the mixture, and the blow and hop kernels alone
    (the two that are ergodic by themselves), reproduce mean 0, variance 1.
"""
import math
import tempfile
from pathlib import Path

import numpy as np
import pytest
from scipy import stats

import oracle

A_W, A_T, N1 = 1.5, 6.0, 4.0


def _proposals(n, count, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for it in range(count):
        x = rng.normal(0, 1, n).astype(np.float32)
        xp = rng.normal(0, 1, n).astype(np.float32)
        side, kern, m, y, W = oracle.twalk_propose(x, xp, seed, 0, it)
        h, r = (x, xp) if side == 0 else (xp, x)
        out.append((side, kern, m, h.astype(np.float64), r.astype(np.float64), y.astype(np.float64), W))
    return out


@pytest.fixture(scope="module")
def props():
    return _proposals(6, 40000)


def test_side_and_kernel_frequencies(props):
    sides = np.array([p[0] for p in props])
    kerns = [p[1] for p in props]
    n = len(props)
    assert abs(sides.mean() - 0.5) < 4 * math.sqrt(0.25 / n)
    for name, pr in (("traverse", 0.4918), ("walk", 0.4918), ("blow", 0.0082), ("hop", 0.0082)):
        f = kerns.count(name) / n
        assert abs(f - pr) < 5 * math.sqrt(pr * (1 - pr) / n), (name, f)


def test_subset_size_distribution(props):
    n = 6
    p = min(n, N1) / n
    m = np.array([q[2] for q in props])
    pk = np.array([stats.binom.pmf(k, n, p) for k in range(1, n + 1)])
    pk /= pk.sum()
    obs = np.array([(m == k).sum() for k in range(1, n + 1)])
    chi2 = ((obs - pk * len(m)) ** 2 / (pk * len(m))).sum()
    assert chi2 < stats.chi2.ppf(0.999, n - 1), (obs, pk * len(m))


def _moved(h, y):
    return np.flatnonzero(y != h)


def test_traverse_beta_distribution_and_factor(props):
    a = A_T
    w1 = (a - 1) / (2 * a)

    def cdf(b):
        b = np.asarray(b)
        return np.where(b <= 1, w1 * b ** (a + 1), w1 + (1 - w1) * (1 - b ** (1 - a)))

    betas = []
    for side, kern, m, h, r, y, W in props:
        if kern != "traverse":
            continue
        j = _moved(h, y)
        assert len(j) == m
        k = j[np.argmax(np.abs(r[j] - h[j]))]
        b = float((y[k] - r[k]) / (r[k] - h[k]))
        # one beta moves every selected coordinate (up to the float rounding of y)
        pred = r[j] + b * (r[j] - h[j])
        assert np.all(np.abs(y[j] - pred) <= 1e-6 * (np.abs(pred) + np.abs(r[j]) + 1e-3))
        betas.append(b)
        assert W == pytest.approx((m - 2) * math.log(b), rel=1e-3, abs=1e-5)
    assert stats.kstest(betas, cdf).pvalue > 1e-3


def test_walk_z_distribution_and_factor(props):
    a = A_W
    lo = -a / (1 + a)

    def cdf(z):
        z = np.clip(np.asarray(z), lo, a)
        return (np.sqrt(1 + z) - math.sqrt(1 + lo)) / (math.sqrt(1 + a) - math.sqrt(1 + lo))

    zs = []
    for side, kern, m, h, r, y, W in props:
        if kern != "walk":
            continue
        assert W == 0.0
        j = _moved(h, y)
        ok = np.abs(h[j] - r[j]) > 1e-3
        zs.extend(((y[j] - h[j]) / (h[j] - r[j]))[ok])
    assert stats.kstest(zs, cdf).pvalue > 1e-3


def _rare_kernel(n, name, count, seed):
    """Force proposals of one rare kernel by scanning iterations."""
    rng = np.random.default_rng(seed)
    out = []
    it = 0
    while len(out) < count:
        x = rng.normal(0, 1, n).astype(np.float32)
        xp = rng.normal(0, 1, n).astype(np.float32)
        side, kern, m, y, W = oracle.twalk_propose(x, xp, seed, 0, it)
        it += 1
        if kern == name:
            h, r = (x, xp) if side == 0 else (xp, x)
            out.append((m, h.astype(np.float64), r.astype(np.float64), y.astype(np.float64), W))
    return out


@pytest.mark.parametrize("name", ["blow", "hop"])
def test_blow_and_hop_draws_and_factor(name):
    zs = []
    for m, h, r, y, W in _rare_kernel(5, name, 400, seed=17 if name == "blow" else 19):
        j = _moved(h, y)
        assert len(j) == m
        sf = np.max(np.abs(r[j] - h[j]))
        sb = np.max(np.abs(r[j] - y[j]))
        if name == "blow":
            zs.extend((y[j] - r[j]) / sf)
            want = stats.norm.logpdf(h[j], r[j], sb).sum() - stats.norm.logpdf(y[j], r[j], sf).sum()
        else:
            zs.extend(3 * (y[j] - h[j]) / sf)
            want = stats.norm.logpdf(h[j], y[j], sb / 3).sum() - stats.norm.logpdf(y[j], h[j], sf / 3).sum()
        assert W == pytest.approx(want, rel=1e-6, abs=1e-6)
    assert stats.kstest(zs, "norm").pvalue > 1e-3


@pytest.mark.parametrize("kernels,name", [((0.4918, 0.9836, 0.9918), "mixture"), ((0, 0, 1), "blow"),
                                          ((0, 0, 0), "hop")])
def test_gaussian_target_moments(kernels, name):
    n = 5
    s = oracle.twalk_gauss_run(np.full(n, 0.5, np.float32), np.full(n, -0.3, np.float32), 300000, 11,
                               kernels=kernels)[20000:]
    assert np.abs(s.mean(0)).max() < 0.08, (name, s.mean(0))
    assert np.abs(s.var(0) - 1).max() < 0.08, (name, s.var(0))


MUTANTS = {
    "traverse_factor": ("w = (m - 2) * log(beta);", "w = m * log(beta);"),
    "traverse_beta": ("pow(u2, 1.0 / (TW_AT + 1.0))", "pow(u2, 1.0 / TW_AT)"),
    "walk_z": ("(-1.0 + 2.0 * u + TW_AW * u * u)", "(-1.0 + 2.0 * u)"),
    "blow_sign": ("w = lnorm_phi(n, phi, h, r, sb) - lnorm_phi(n, phi, yr, r, sf);",
                  "w = lnorm_phi(n, phi, yr, r, sf) - lnorm_phi(n, phi, h, r, sb);"),
    "hop_sigma": ("w = lnorm_phi(n, phi, h, yr, sb / 3.0) - lnorm_phi(n, phi, yr, h, sf / 3.0);",
                  "w = lnorm_phi(n, phi, h, yr, sf / 3.0) - lnorm_phi(n, phi, yr, h, sf / 3.0);"),
    "blow_center": ("(blow ? r[j] : h[j]) + s *", "h[j] + s *"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, monkeypatch):
    """Each planted mistake fails at least one of the pins above."""
    here = Path(oracle.__file__).parent
    base = (here / "mcmc_oracle.c").read_text()
    tw = (here / "twalk_oracle.c").read_text()
    a, b = MUTANTS[name]
    assert a in tw
    L = oracle.compile_variant(base + "\n" + tw.replace(a, b), tempfile.mkdtemp())
    monkeypatch.setattr(oracle, "lib", lambda: L)
    caught = []
    props = _proposals(6, 40000)
    for pin in (lambda: test_walk_z_distribution_and_factor(props),
                lambda: test_traverse_beta_distribution_and_factor(props),
                lambda: test_blow_and_hop_draws_and_factor("blow"),
                lambda: test_blow_and_hop_draws_and_factor("hop")):
        try:
            pin()
        except AssertionError:
            caught.append(True)
    assert caught, name
