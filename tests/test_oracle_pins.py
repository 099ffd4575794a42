"""Pins for the CPU oracle, from what the paper and the mathematics fix.

The paper prints no worked log-likelihood values, so the oracle is pinned
constructively (each test names the passage it follows):

* brute-force summation over all K^T hidden paths (Eq. "likelihood func");
* closed forms: T = 1, identical transition rows (a product of mixture
  densities), P = I, K = 1, T = 0;
* invariants: label permutation, time reversal of a reversible chain,
  coordinate rescaling, segment additivity, the two initial conventions
  agreeing when pi is stationary;
* the emission of Eq. "emission-matrix" against scipy's bivariate normal,
  its peak value, its integral by quadrature, and its factorisation at rho=0;
* the oracle's own rounding: an independent backward recursion and a
  long-double run.

Reference values in the closed-form tests are computed here with numpy/scipy
from the formulas, not by calling the oracle.
"""
import math

import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

import oracle
from paper_2003_03508_gb300 import synth


def _logemis_scipy(prm, x, y, flag):
    """log e_k(o) from scipy's bivariate normal (Eq. "emission-matrix")."""
    K = prm.K
    out = np.empty(K)
    for k in range(K):
        p = float(prm.p_tremor[k])
        if not flag:
            out[k] = math.log1p(-p) if p < 1 else -math.inf
            continue
        c = prm.cov[k].astype(np.float64)
        S = np.array([[c[0], c[1]], [c[1], c[2]]])
        out[k] = (math.log(p) if p > 0 else -math.inf) + multivariate_normal(
            mean=prm.mu[k].astype(np.float64), cov=S).logpdf([float(x), float(y)])
    return out


def _small(K, T, seed, **kw):
    rng = np.random.default_rng(seed)
    prm = synth.random_params(K, rng, **kw)
    obs = synth.sample_observations(prm, T, rng)
    return prm, obs


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("T", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("init_mode", [0, 1])
def test_bruteforce_K3(T, seed, init_mode):
    # Eq. "likelihood func": sum over all 3^T paths, vs the scaled recursion
    prm, obs = _small(3, T, 100 + seed, diag=(0.3, 0.9))
    # a non-symmetric, non-stationary chain so a transposed P or a wrong
    # initial convention cannot pass
    bf = oracle.loglik_bruteforce(prm, obs.xy, obs.tremor, init_mode)
    fw = oracle.loglik(prm, obs.xy, obs.tremor, init_mode)
    assert math.isfinite(bf)
    assert abs(fw - bf) <= 1e-13 * max(1.0, abs(bf)), (fw, bf)


def test_bruteforce_mixed_flags_K4():
    rng = np.random.default_rng(7)
    prm = synth.random_params(4, rng, diag=(0.2, 0.6))
    xy = rng.uniform(0, 150, size=(7, 2)).astype(np.float32)
    flags = np.array([1, 0, 1, 1, 0, 1, 0], np.uint8)
    bf = oracle.loglik_bruteforce(prm, xy, flags)
    fw = oracle.loglik(prm, xy, flags)
    assert abs(fw - bf) <= 1e-13 * abs(bf)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("flag", [0, 1])
@pytest.mark.parametrize("init_mode", [0, 1])
def test_T1_closed_form(flag, init_mode):
    # T = 1: L = pi0^T e(o_1) with pi0 = pi (emit first) or P^T pi
    rng = np.random.default_rng(11)
    prm = synth.random_params(6, rng)
    prm.pi[:] = rng.dirichlet(np.ones(6)).astype(np.float32)
    x, y = 120.5, 64.25
    le = _logemis_scipy(prm, x, y, flag)
    pi0 = prm.pi.astype(np.float64)
    if init_mode == 1:
        pi0 = prm.P.astype(np.float64).T @ pi0
    ref = logsumexp(np.log(pi0) + le)
    got = oracle.loglik(prm, np.array([[x, y]], np.float32), np.array([flag], np.uint8), init_mode)
    assert abs(got - ref) <= 1e-12 * max(1, abs(ref))


def test_identical_rows_mixture_product():
    # P = 1 w^T: the hidden states are iid w after the first, so
    # log L = log(pi^T e(o_1)) + sum_{t>=2} log(w^T e(o_t))
    rng = np.random.default_rng(12)
    K, T = 7, 400
    prm = synth.random_params(K, rng)
    w = rng.dirichlet(np.ones(K))
    prm.P[:] = np.tile(w.astype(np.float32), (K, 1))
    prm.pi[:] = rng.dirichlet(np.ones(K)).astype(np.float32)
    obs = synth.sample_observations(prm, T, rng)
    wf = prm.P[0].astype(np.float64)
    ref = 0.0
    for t in range(T):
        le = _logemis_scipy(prm, obs.xy[t, 0], obs.xy[t, 1], obs.tremor[t])
        ref += logsumexp((np.log(prm.pi.astype(np.float64)) if t == 0 else np.log(wf)) + le)
    got = oracle.loglik(prm, obs.xy, obs.tremor)
    assert abs(got - ref) <= 1e-11 * abs(ref), (got, ref)


def test_identity_transition():
    # P = I: the state never changes, L = sum_k pi_k prod_t e_k(o_t)
    rng = np.random.default_rng(13)
    K, T = 5, 300
    prm = synth.random_params(K, rng)
    prm.P[:] = np.eye(K, dtype=np.float32)
    prm.pi[:] = rng.dirichlet(np.ones(K)).astype(np.float32)
    xy = rng.uniform(0, 200, size=(T, 2)).astype(np.float32)
    fl = (rng.random(T) < 0.4).astype(np.uint8)
    S = np.zeros(K)
    for t in range(T):
        S += _logemis_scipy(prm, xy[t, 0], xy[t, 1], fl[t])
    ref = logsumexp(np.log(prm.pi.astype(np.float64)) + S)
    got = oracle.loglik(prm, xy, fl)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_single_state():
    # K = 1: log L = sum_t log e_1(o_t)
    rng = np.random.default_rng(14)
    prm = synth.random_params(1, rng)
    xy = rng.uniform(0, 300, size=(1000, 2)).astype(np.float32)
    fl = (rng.random(1000) < 0.5).astype(np.uint8)
    ref = sum(_logemis_scipy(prm, xy[t, 0], xy[t, 1], fl[t])[0] for t in range(1000))
    got = oracle.loglik(prm, xy, fl)
    assert abs(got - ref) <= 1e-11 * abs(ref)


def test_empty_sequence():
    prm, _ = _small(4, 1, 0)
    e = np.zeros((0, 2), np.float32)
    f = np.zeros(0, np.uint8)
    assert abs(oracle.loglik(prm, e, f) - math.log(float(prm.pi.astype(np.float64).sum()))) < 1e-15
    assert oracle.loglik_backward(prm, e, f) == pytest.approx(oracle.loglik(prm, e, f), abs=1e-15)


def test_zero_likelihood_is_minus_inf():
    # every state has p_k = 0 and a tremor is observed: L = 0 exactly
    prm, obs = _small(3, 20, 5)
    prm.p_tremor[:] = 0.0
    fl = obs.tremor.copy()
    fl[:] = 0
    fl[10] = 1
    assert oracle.loglik(prm, obs.xy, fl) == -math.inf
    assert oracle.loglik_backward(prm, obs.xy, fl) == -math.inf
    assert oracle.loglik_bruteforce(prm, obs.xy[:6], fl[:6]) > -math.inf  # no tremor in first 6
    fl2 = fl[:6].copy(); fl2[3] = 1
    assert oracle.loglik_bruteforce(prm, obs.xy[:6], fl2) == -math.inf


# ---------------------------------------------------------------- invariants

def test_label_permutation():
    prm, obs = _small(6, 2000, 21)
    perm = np.random.default_rng(3).permutation(6)
    q = synth.HMMParams(prm.pi[perm].copy(), prm.P[np.ix_(perm, perm)].copy(),
                        prm.p_tremor[perm].copy(), prm.mu[perm].copy(), prm.cov[perm].copy())
    a = oracle.loglik(prm, obs.xy, obs.tremor)
    b = oracle.loglik(q, obs.xy, obs.tremor)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_time_reversal_reversible_chain():
    # P from a symmetric weight matrix W (P_ij = W_ij / sum_j W_ij) is
    # reversible w.r.t. pi_i proportional to the row sums, so the reversed
    # sequence has the same likelihood when started from that pi.
    rng = np.random.default_rng(22)
    K, T = 5, 500
    W = rng.uniform(0.1, 1.0, size=(K, K))
    W = W + W.T + np.diag(rng.uniform(2, 6, K))
    prm = synth.random_params(K, rng)
    prm.P[:] = (W / W.sum(1, keepdims=True)).astype(np.float32)
    # stationary distribution of the float32 P (to double precision)
    P64 = prm.P.astype(np.float64)
    evals, evecs = np.linalg.eig(P64.T)
    v = np.real(evecs[:, np.argmin(abs(evals - 1))])
    pi = v / v.sum()
    obs = synth.sample_observations(prm, T, rng)
    # pass pi via double-accurate float32 rounding: small residual is allowed below
    prm.pi[:] = pi.astype(np.float32)
    fwd = oracle.loglik(prm, obs.xy, obs.tremor)
    rev = oracle.loglik(prm, obs.xy[::-1].copy(), obs.tremor[::-1].copy())
    # float32 P is only approximately reversible: detailed balance holds to ~1e-7
    assert abs(fwd - rev) <= 5e-4 * T * 1e-3 + 1e-5 * abs(fwd)


def test_coordinate_rescale():
    # x -> s x, mu -> s mu, Sigma -> s^2 Sigma scales each tremor density by
    # 1/s^2, so log L changes by exactly -2 n_tremor log s (s = 2: exact in fp32)
    prm, obs = _small(5, 3000, 23)
    s = 2.0
    q = synth.HMMParams(prm.pi, prm.P, prm.p_tremor, prm.mu * s, prm.cov * s * s)
    a = oracle.loglik(prm, obs.xy, obs.tremor)
    b = oracle.loglik(q, obs.xy * s, obs.tremor)
    n = int(obs.tremor.sum())
    assert abs((b - a) - (-2.0 * n * math.log(s))) <= 1e-9 * abs(a)


def test_segment_additivity_and_batch():
    rng = np.random.default_rng(24)
    gen = synth.random_params(4, rng)
    lens = [37, 1, 400, 2, 1000]
    xy, fl, offs = synth.sample_segments(gen, lens, rng)
    props = [synth.perturb_params(gen, rng) for _ in range(3)]
    st = synth.stack_params(props)
    got = oracle.loglik_batched(st, xy, fl, offs, n_threads=2)
    for q in range(3):
        ref = 0.0   # plain left-to-right sum (Python's sum() is compensated)
        for s in range(len(lens)):
            ref += oracle.loglik(props[q], xy[offs[s]:offs[s + 1]], fl[offs[s]:offs[s + 1]])
        assert got[q] == ref


def test_stationary_init_conventions_agree():
    # Eq. "likelihood func" applies Gamma before the first emission; with a
    # stationary pi both conventions give the same L
    prm, obs = _small(4, 800, 25)
    P64 = prm.P.astype(np.float64)
    evals, evecs = np.linalg.eig(P64.T)
    v = np.real(evecs[:, np.argmin(abs(evals - 1))])
    prm.pi[:] = (v / v.sum()).astype(np.float32)
    a = oracle.loglik(prm, obs.xy, obs.tremor, 0)
    b = oracle.loglik(prm, obs.xy, obs.tremor, 1)
    assert abs(a - b) <= 1e-6   # pi is stationary only to float32 rounding
    prm.pi[:] = np.float32([1, 0, 0, 0])
    assert abs(oracle.loglik(prm, obs.xy, obs.tremor, 0) -
               oracle.loglik(prm, obs.xy, obs.tremor, 1)) > 1e-3


# ---------------------------------------------------------------- emission

def test_emission_matches_scipy():
    rng = np.random.default_rng(31)
    prm = synth.random_params(9, rng)
    for _ in range(20):
        x, y = float(np.float32(rng.uniform(-50, 350))), float(np.float32(rng.uniform(-50, 200)))
        for flag in (0, 1):
            a = oracle.log_emission(prm, x, y, flag)
            b = _logemis_scipy(prm, x, y, flag)
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_emission_peak_and_quadrature():
    rng = np.random.default_rng(32)
    prm = synth.random_params(3, rng)
    prm.p_tremor[:] = 1.0
    for k in range(3):
        c = prm.cov[k].astype(np.float64)
        det = c[0] * c[2] - c[1] ** 2
        le = oracle.log_emission(prm, float(prm.mu[k, 0]), float(prm.mu[k, 1]), 1)
        assert abs(le[k] - (-math.log(2 * math.pi * math.sqrt(det)))) < 1e-12
        # integral of phi over a +-8 sigma grid
        sx, sy = math.sqrt(c[0]), math.sqrt(c[2])
        gx = np.linspace(prm.mu[k, 0] - 8 * sx, prm.mu[k, 0] + 8 * sx, 401)
        gy = np.linspace(prm.mu[k, 1] - 8 * sy, prm.mu[k, 1] + 8 * sy, 401)
        dens = np.array([[math.exp(oracle.log_emission(prm, x, y, 1)[k]) for x in gx] for y in gy])
        integ = np.trapezoid(np.trapezoid(dens, gx, axis=1), gy)
        assert abs(integ - 1.0) < 1e-6


def test_emission_rho0_factorises():
    rng = np.random.default_rng(33)
    prm = synth.random_params(4, rng)
    prm.cov[:, 1] = 0.0
    x, y = 101.0, 77.0
    le = oracle.log_emission(prm, x, y, 1)
    for k in range(4):
        sx, sy = math.sqrt(float(prm.cov[k, 0])), math.sqrt(float(prm.cov[k, 2]))
        mx, my = float(prm.mu[k, 0]), float(prm.mu[k, 1])
        nx = -0.5 * math.log(2 * math.pi) - math.log(sx) - 0.5 * ((x - mx) / sx) ** 2
        ny = -0.5 * math.log(2 * math.pi) - math.log(sy) - 0.5 * ((y - my) / sy) ** 2
        assert abs(le[k] - (math.log(float(prm.p_tremor[k])) + nx + ny)) < 1e-11


# ---------------------------------------------------------------- rounding

def test_forward_backward_and_longdouble_k4_t1e4():
    d = synth.config_inputs("k4_t1e4")
    a = oracle.loglik(d["params"], d["xy"], d["tremor"])
    b = oracle.loglik_backward(d["params"], d["xy"], d["tremor"])
    c = oracle.loglik_longdouble(d["params"], d["xy"], d["tremor"])
    assert abs(a - b) <= 1e-12 * abs(a)
    assert abs(a - c) <= 1e-12 * abs(a)


def test_longdouble_k25_t1e5():
    rng = np.random.default_rng(41)
    prm = synth.quiescent_params(25, rng)
    obs = synth.sample_observations(prm, 100_000, rng)
    a = oracle.loglik(prm, obs.xy, obs.tremor)
    c = oracle.loglik_longdouble(prm, obs.xy, obs.tremor)
    assert abs(a - c) <= 1e-12 * abs(a)
