"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each mutant is the oracle source with one edit (a transposed operand, a
dropped term, a flipped sign, a wrong initial convention, an index slip),
compiled on the CPU. The independent pins -- brute force over paths,
the T = 1 closed form from scipy's bivariate normal, the identical-rows
mixture product and the P = I closed form -- must reject every mutant, and
accept the unmodified source.
"""
import math
from pathlib import Path

import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

import oracle
from paper_2003_03508_gb300 import synth

SRC = (Path(oracle.__file__).parent / "hmm_oracle.c").read_text()

MUTANTS = {
    "transposed_P": ("s += alpha[i] * (double)P[i * K + j];", "s += alpha[i] * (double)P[j * K + i];"),
    "dropped_logdet": ("- 0.5 * log(det) - 0.5 * q;", "- 0.5 * q;"),
    "sign_sxy": ("q = (syy * dx * dx - 2.0 * sxy * dx * dy", "q = (syy * dx * dx + 2.0 * sxy * dx * dy"),
    "swapped_mu": ("double dx = x - (double)mu[2 * k + 0];", "double dx = x - (double)mu[2 * k + 1];"),
    "init_convention": ("if (init_mode == 1) {           /* delta^T Gamma",
                        "if (init_mode == 0) {           /* delta^T Gamma"),
    "dropped_log_c": ("double term = m + log(c);", "double term = m;"),
    "wrong_no_tremor": ("out[k] = log(1.0 - pk);", "out[k] = log(pk);"),
    "skipped_first_transition": ("if (t == 0) {\n            for (int k = 0; k < K; ++k) beta[k] = alpha[k];",
                                 "if (t <= 1) {\n            for (int k = 0; k < K; ++k) beta[k] = alpha[k];"),
}


def _scipy_le(prm, x, y, flag):
    out = np.empty(prm.K)
    for k in range(prm.K):
        p = float(prm.p_tremor[k])
        if not flag:
            out[k] = math.log1p(-p)
            continue
        c = prm.cov[k].astype(np.float64)
        out[k] = math.log(p) + multivariate_normal(
            mean=prm.mu[k].astype(np.float64),
            cov=[[c[0], c[1]], [c[1], c[2]]]).logpdf([float(x), float(y)])
    return out


def _pins_pass(L) -> bool:
    rng = np.random.default_rng(5)
    # 1. brute force, non-symmetric chain, both conventions
    prm = synth.random_params(3, rng, diag=(0.3, 0.8))
    prm.pi[:] = np.float32([0.6, 0.3, 0.1])
    obs = synth.sample_observations(prm, 6, rng)
    for mode in (0, 1):
        bf = oracle.loglik_bruteforce(prm, obs.xy, obs.tremor, mode)
        fw = oracle.loglik(prm, obs.xy, obs.tremor, mode, _L=L)
        if not abs(fw - bf) <= 1e-12 * abs(bf):
            return False
        ref_bf = oracle.loglik_bruteforce(prm, obs.xy, obs.tremor, mode, _L=L)
        if not abs(ref_bf - bf) <= 1e-12 * abs(bf):
            return False
    # 2. T = 1 closed forms, both flags and conventions
    for flag in (0, 1):
        x, y = 101.5, 52.25
        le = _scipy_le(prm, x, y, flag)
        for mode in (0, 1):
            pi0 = prm.pi.astype(np.float64)
            if mode == 1:
                pi0 = prm.P.astype(np.float64).T @ pi0
            ref = logsumexp(np.log(pi0) + le)
            got = oracle.loglik(prm, np.float32([[x, y]]), np.uint8([flag]), mode, _L=L)
            if not abs(got - ref) <= 1e-12 * max(1, abs(ref)):
                return False
    # 3. identical rows
    K = 4
    q = synth.random_params(K, rng)
    w = rng.dirichlet(np.ones(K)).astype(np.float32)
    q.P[:] = np.tile(w, (K, 1))
    o = synth.sample_observations(q, 50, rng)
    ref = 0.0
    for t in range(50):
        le = _scipy_le(q, o.xy[t, 0], o.xy[t, 1], o.tremor[t])
        ref += logsumexp((np.log(q.pi.astype(np.float64)) if t == 0 else np.log(w.astype(np.float64))) + le)
    if not abs(oracle.loglik(q, o.xy, o.tremor, _L=L) - ref) <= 1e-11 * abs(ref):
        return False
    return True


def test_unmodified_source_passes(tmp_path):
    L = oracle.compile_variant(SRC, tmp_path)
    assert _pins_pass(L)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    assert SRC.count(old) >= 1, f"mutation anchor for {name} not found"
    L = oracle.compile_variant(SRC.replace(old, new, 1), tmp_path)
    assert not _pins_pass(L), f"pins did not catch mutant {name}"
