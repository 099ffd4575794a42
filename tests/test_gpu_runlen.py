"""Parity of the run-length shortcut (opts.runlen_min > 0) with the FP64 oracle.

The shortcut computes the same likelihood (a run of n no-tremor steps
contributes (P D_0)^n, formed from binary powers), so the oracle is the
plain forward algorithm and the bar is the FP32 one:
  |d| <= 1e-6 |log L| + 1e-4.
Cases: every K the FP32 path supports, run lengths that cross chunk
boundaries and the ragged tail, several thresholds, reducible P (rows of
(P D_0)^n decaying at rates far apart), a state that always emits a tremor
(a zero column in D_0), sequences with no tremor at all, zero likelihood,
batched ragged segments, and the full-size batched workload on sampled
proposals.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_REL, FP32_ABS = 1e-6, 1e-4


def _close(got, ref, rel=FP32_REL, ab=FP32_ABS):
    if ref == -math.inf:
        return got == -math.inf
    return abs(got - ref) <= rel * abs(ref) + ab


def _gpu(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    t = api.to_device(prm)
    xy_d = torch.from_numpy(np.ascontiguousarray(xy, np.float32).reshape(-1, 2)).cuda()
    fl_d = torch.from_numpy(np.ascontiguousarray(tremor, np.uint8)).cuda()
    out = ctx.hmm_loglik(*t, xy_d, fl_d, opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return float(out.item())


def _runs(tremor):
    """Lengths of the maximal runs of no-tremor steps after the first step."""
    z = np.concatenate([[1], np.asarray(tremor[1:], np.int64), [1]])
    idx = np.flatnonzero(z)
    return np.diff(idx) - 1


@pytest.mark.parametrize("K", [1, 2, 3, 7, 16, 25, 32, 33, 48, 64, 80])
def test_parity_sizes(cuda_lib, K):
    rng = np.random.default_rng(3100 + K)
    prm = synth.random_params(K, rng, p_range=synth.SPARSE_P_RANGE)
    T = 20_000 + 37
    obs = synth.sample_observations(prm, T, rng)
    assert _runs(obs.tremor).max() > 64  # runs longer than the shortest chunks
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    for L, n_min in ((256, 1), (256, 4), (64, 64), (0, 4)):
        got = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=L, runlen_min=n_min)
        assert _close(got, ref), (K, L, n_min, got, ref)


@pytest.mark.parametrize("init_mode", [0, 1])
def test_init_modes(cuda_lib, init_mode):
    rng = np.random.default_rng(3200 + init_mode)
    prm = synth.random_params(9, rng, p_range=synth.SPARSE_P_RANGE)
    obs = synth.sample_observations(prm, 30_001, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor, init_mode)
    got = _gpu(cuda_lib, prm, obs.xy, obs.tremor, init_mode=init_mode, chunk_len=512, runlen_min=2)
    assert _close(got, ref), (got, ref)


@pytest.mark.parametrize("T", [1, 2, 3, 64, 65, 1000, 65_537])
def test_no_tremor_at_all(cuda_lib, T):
    # one run covering everything after the first step, cut by the chunks
    rng = np.random.default_rng(3300 + T)
    prm = synth.random_params(6, rng)
    xy = np.zeros((T, 2), np.float32)
    fl = np.zeros(T, np.uint8)
    ref = oracle.loglik(prm, xy, fl)
    for L in (64, 0):
        got = _gpu(cuda_lib, prm, xy, fl, chunk_len=L, runlen_min=1)
        assert _close(got, ref), (T, L, got, ref)


def _by_groups(prm, groups, xy, tremor):
    """log L of a chain whose states split into closed groups (P is block
    diagonal): L = sum_g pi(g) L_g, L_g the likelihood of the sub-chain on g
    started from pi restricted to g and renormalised. Each L_g comes from the
    oracle on a connected chain. (The oracle's per-step scaling cannot be
    used on the whole chain here: it flushes a group whose forward
    probability falls below 2^-1074 of the leading one, and a group that is
    behind early can lead later.)"""
    out = []
    for g in groups:
        g = np.asarray(g)
        pg = float(prm.pi[g].astype(np.float64).sum())
        sub = synth.HMMParams((prm.pi[g] / np.float32(pg)).astype(np.float32),
                              prm.P[np.ix_(g, g)].copy(), prm.p_tremor[g].copy(), prm.mu[g].copy(),
                              prm.cov[g].copy())
        out.append(math.log(pg) + oracle.loglik(sub, xy, tremor))
    m = max(out)
    return m + math.log(sum(math.exp(v - m) for v in out))


def test_reducible_transitions(cuda_lib):
    # P = I: state k's rows of (P D_0)^n decay like (1 - p_k)^n, 0.1^n next to
    # 0.999^n, far outside one float exponent range; each table row keeps its
    # own exponent. Every state emits tremors at the same place, so no state
    # is flushed at a tremor step (each step scales by its best state's power
    # of two; with P = I a row holds one state only).
    rng = np.random.default_rng(3400)
    K = 4
    prm = synth.random_params(K, rng)
    prm.P[:] = np.eye(K, dtype=np.float32)
    prm.p_tremor[:] = np.array([0.9, 0.001, 0.5, 0.02], np.float32)
    prm.mu[:] = (150.0, 75.0)
    prm.cov[:] = (100.0, 0.0, 100.0)
    T = 40_000
    fl = np.zeros(T, np.uint8)
    fl[rng.choice(T, 300, replace=False)] = 1
    fl[:1025] = 1  # the first chunk favours p = 0.9, the whole p = 0.02
    xy = np.where(fl[:, None] == 1, rng.normal((150.0, 75.0), 10.0, (T, 2)), 0.0).astype(np.float32)
    ref = _by_groups(prm, [[0], [1], [2], [3]], xy, fl)
    # closed form of the P = I chain: log sum_k pi_k p_k^n1 (1 - p_k)^n0 + sum log N(o_t)
    p = prm.p_tremor.astype(np.float64)
    n1 = int(fl.sum())
    terms = np.log(prm.pi.astype(np.float64)) + n1 * np.log(p) + (T - n1) * np.log1p(-p)
    dd = xy[fl == 1].astype(np.float64) - (150.0, 75.0)
    lg = -np.log(2 * np.pi * 100.0) - 0.5 * (dd ** 2).sum(axis=1) / 100.0
    want = terms.max() + math.log(np.exp(terms - terms.max()).sum()) + lg.sum()
    assert abs(ref - want) < 1e-9 * abs(want), (ref, want)
    for L in (1024, 64, 0):
        got = _gpu(cuda_lib, prm, xy, fl, chunk_len=L, runlen_min=1)
        assert _close(got, ref), (L, got, ref)
    # block-diagonal P: two groups that never mix; the data favour the
    # tremor-rich group first and the quiet group overall
    prm2 = synth.random_params(K, rng)
    P = np.zeros((K, K))
    P[:2, :2] = [[0.97, 0.03], [0.05, 0.95]]
    P[2:, 2:] = [[0.9, 0.1], [0.2, 0.8]]
    prm2.P[:] = P.astype(np.float32)
    prm2.p_tremor[:] = np.array([0.6, 0.7, 0.002, 0.01], np.float32)
    prm2.mu[:] = (150.0, 75.0)
    prm2.cov[:] = (100.0, 0.0, 100.0)
    ref = _by_groups(prm2, [[0, 1], [2, 3]], xy, fl)
    for L in (2048, 0):
        got = _gpu(cuda_lib, prm2, xy, fl, chunk_len=L, runlen_min=3)
        assert _close(got, ref), (L, got, ref)


def test_state_that_always_emits(cuda_lib):
    # p_k = 1: D_0 has a zero entry, so that state's column of every power is zero
    rng = np.random.default_rng(3500)
    prm = synth.random_params(5, rng, p_range=synth.SPARSE_P_RANGE)
    prm.p_tremor[2] = 1.0
    obs = synth.sample_observations(prm, 10_000, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    got = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=256, runlen_min=1)
    assert _close(got, ref), (got, ref)


def test_zero_likelihood(cuda_lib):
    # every state always emits a tremor: a no-tremor run has probability zero
    rng = np.random.default_rng(3600)
    prm = synth.random_params(3, rng)
    prm.p_tremor[:] = 1.0
    xy = np.zeros((500, 2), np.float32)
    fl = np.zeros(500, np.uint8)
    fl[0] = 1
    assert oracle.loglik(prm, xy, fl) == -math.inf
    assert _gpu(cuda_lib, prm, xy, fl, chunk_len=64, runlen_min=1) == -math.inf


def test_same_as_without_the_shortcut(cuda_lib):
    rng = np.random.default_rng(3700)
    prm = synth.random_params(32, rng, p_range=synth.SPARSE_P_RANGE)
    obs = synth.sample_observations(prm, 100_000, rng)
    a = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=1024)
    b = _gpu(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=1024, runlen_min=4)
    assert abs(a - b) <= 2e-7 * abs(a), (a, b)
    # the random workload (short runs) gives the same answer too
    prm = synth.random_params(32, rng)
    obs = synth.sample_observations(prm, 50_000, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    assert _close(_gpu(cuda_lib, prm, obs.xy, obs.tremor, runlen_min=2), ref)


def test_batched_ragged_segments(cuda_lib):
    api = cuda_lib
    d = synth.batched_inputs(K=12, T=80_000, n_prop=6, seed=37, n_seg=9, sparse=True)
    ctx = api.default_context()
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    got = ctx.hmm_loglik_batched(*api.to_device(d["params"]), d["offsets"], xy, fl,
                                 opts=api.make_opts(chunk_len=512, runlen_min=4)).cpu().numpy()
    ref = oracle.loglik_batched(d["params"], d["xy"], d["tremor"], d["offsets"], n_threads=4)
    for q in range(len(ref)):
        assert _close(float(got[q]), float(ref[q])), (q, got[q], ref[q])


def test_option_errors(cuda_lib):
    api = cuda_lib
    rng = np.random.default_rng(3800)
    prm = synth.random_params(8, rng)
    obs = synth.sample_observations(prm, 1000, rng)
    with pytest.raises(api.HMMError) as e:
        _gpu(api, prm, obs.xy, obs.tremor, precision="tf32", runlen_min=4)
    assert e.value.code == api.HMM_EUNSUPPORTED
    for bad in (-1, 16385):
        with pytest.raises(api.HMMError) as e:
            _gpu(api, prm, obs.xy, obs.tremor, runlen_min=bad)
        assert e.value.code == api.HMM_EINVAL


def test_full_size_sampled(cuda_lib):
    # the sparse-tremor workload at the likelihood benchmark's size:
    # K = 32, T = 2^20, 256 proposals; the oracle checks 6 of them
    api = cuda_lib
    d = synth.batched_inputs(K=32, T=1 << 20, n_prop=256, seed=41, sparse=True)
    ctx = api.default_context()
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    got = ctx.hmm_loglik_batched(*api.to_device(d["params"]), d["offsets"], xy, fl,
                                 opts=api.make_opts(runlen_min=4)).cpu().numpy()
    assert np.all(np.isfinite(got))
    pick = [0, 1, 77, 128, 200, 255]
    sub = synth.HMMParams(*(a[pick] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=6)
    for j, q in enumerate(pick):
        assert _close(float(got[q]), float(ref[j])), (q, got[q], ref[j])


def test_sparse_workload_tf32_split(cuda_lib):
    # Tensor cores on the sparse-tremor workload: |log L| per step is ~13x
    # smaller than on the random workload, so TF32's rounding of P (a per-step
    # bias in log of up to ~1e-4) leaves the 1e-4 relative bar (2.6e-4
    # measured); with P as TF32 hi + lo the bar holds (5e-6 measured).
    api = cuda_lib
    d = synth.batched_inputs(K=32, T=1 << 20, n_prop=64, seed=43, sparse=True)
    ctx = api.default_context()
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    got = ctx.hmm_loglik_batched(*api.to_device(d["params"]), d["offsets"], xy, fl,
                                 opts=api.make_opts(precision="tf32_split")).cpu().numpy()
    pick = [0, 31, 63]
    sub = synth.HMMParams(*(a[pick] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=3)
    rel = np.abs(got[pick] - ref) / np.abs(ref)
    print("tf32_split sparse rel err", rel)
    assert np.all(rel <= 1e-4), rel
