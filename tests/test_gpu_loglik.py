"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative to the oracle's log L, with an absolute floor for tiny
sequences whose |log L| is O(1)):
  FP32-SIMT chunk products:  |d| <= 1e-6 |log L| + 1e-4
The per-T budget behind them is derived in the design notes: FP32 rounding of
the running product contributes O(sqrt(T) u) with u = 2^-24, and the FP32
emission constants a bias of O(T u |log e|); both are far inside 1e-6 |log L|
at every size tested.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_REL, FP32_ABS = 1e-6, 1e-4


def _gpu_loglik(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    t = api.to_device(prm)
    xy_d = torch.from_numpy(np.ascontiguousarray(xy, np.float32).reshape(-1, 2)).cuda()
    fl_d = torch.from_numpy(np.ascontiguousarray(tremor, np.uint8)).cuda()
    out = ctx.hmm_loglik(*t, xy_d, fl_d, opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return float(out.item())


def _close(got, ref, rel=FP32_REL, ab=FP32_ABS):
    if ref == -math.inf:
        return got == -math.inf
    return abs(got - ref) <= rel * abs(ref) + ab


@pytest.mark.parametrize("K", [1, 2, 3, 4, 7, 16, 25, 32, 33, 48, 64, 80])
def test_fp32_parity_sizes(cuda_lib, K):
    # several chunks and a ragged tail: T not a multiple of the chunk length
    rng = np.random.default_rng(1000 + K)
    prm = synth.random_params(K, rng)
    T = 5000 + 37
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    for L in (64, 256, 0):
        got = _gpu_loglik(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=L)
        assert _close(got, ref), (K, L, got, ref)


@pytest.mark.parametrize("T", [0, 1, 2, 3, 63, 64, 65, 66, 127, 129])
def test_fp32_small_T(cuda_lib, T):
    rng = np.random.default_rng(77 + T)
    prm = synth.random_params(5, rng)
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    got = _gpu_loglik(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=64)
    assert _close(got, ref), (T, got, ref)


@pytest.mark.parametrize("init_mode", [0, 1])
def test_init_modes(cuda_lib, init_mode):
    rng = np.random.default_rng(5)
    prm = synth.random_params(6, rng, diag=(0.5, 0.9))
    prm.pi[:] = np.float32([0.5, 0.2, 0.1, 0.1, 0.05, 0.05])
    obs = synth.sample_observations(prm, 3000, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor, init_mode)
    got = _gpu_loglik(cuda_lib, prm, obs.xy, obs.tremor, init_mode=init_mode, chunk_len=128)
    assert _close(got, ref)


def test_k4_t1e4(cuda_lib):
    d = synth.config_inputs("k4_t1e4")
    ref = oracle.loglik(d["params"], d["xy"], d["tremor"])
    got = _gpu_loglik(cuda_lib, d["params"], d["xy"], d["tremor"])
    assert _close(got, ref), (got, ref)


def test_k25_t2p20_fp32(cuda_lib):
    d = synth.config_inputs("k25_t2p20")
    ref = oracle.loglik(d["params"], d["xy"], d["tremor"])
    got = _gpu_loglik(cuda_lib, d["params"], d["xy"], d["tremor"])
    assert abs(got - ref) <= FP32_REL * abs(ref), (got, ref, (got - ref) / ref)


def test_bit_reproducible(cuda_lib):
    d = synth.config_inputs("k4_t1e4")
    a = _gpu_loglik(cuda_lib, d["params"], d["xy"], d["tremor"])
    b = _gpu_loglik(cuda_lib, d["params"], d["xy"], d["tremor"])
    assert a == b


def test_renorm_interval_invariance(cuda_lib):
    rng = np.random.default_rng(9)
    prm = synth.random_params(12, rng)
    obs = synth.sample_observations(prm, 4000, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    vals = [_gpu_loglik(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=256, renorm_every=r)
            for r in (1, 2, 4, 8)]
    for v in vals:
        assert _close(v, ref)


def test_zero_likelihood(cuda_lib):
    rng = np.random.default_rng(3)
    prm = synth.random_params(4, rng)
    prm.p_tremor[:] = 0.0
    xy = np.zeros((500, 2), np.float32)
    fl = np.zeros(500, np.uint8)
    fl[321] = 1
    xy[321] = (10.0, 20.0)
    assert oracle.loglik(prm, xy, fl) == -math.inf
    assert _gpu_loglik(cuda_lib, prm, xy, fl, chunk_len=64) == -math.inf
    fl[321] = 0
    ref = oracle.loglik(prm, xy, fl)
    assert _close(_gpu_loglik(cuda_lib, prm, xy, fl, chunk_len=64), ref)


def test_invalid_params_give_nan_and_einval(cuda_lib):
    api = cuda_lib
    ctx = api.default_context()
    ctx.hmm_status()  # clear
    rng = np.random.default_rng(4)
    prm = synth.random_params(4, rng)
    obs = synth.sample_observations(prm, 100, rng)
    bad = synth.HMMParams(prm.pi.copy(), prm.P.copy(), prm.p_tremor.copy(), prm.mu.copy(), prm.cov.copy())
    bad.P[1, 1] += 0.01  # row no longer sums to 1
    got = _gpu_loglik(api, bad, obs.xy, obs.tremor)
    assert math.isnan(got)
    assert ctx.hmm_status() == api.HMM_EINVAL
    assert ctx.hmm_status() == api.HMM_OK  # cleared by the read
    bad2 = synth.HMMParams(prm.pi, prm.P, prm.p_tremor, prm.mu, prm.cov.copy())
    bad2.cov[2] = (1.0, 2.0, 1.0)  # not positive definite
    assert math.isnan(_gpu_loglik(api, bad2, obs.xy, obs.tremor))
    assert ctx.hmm_status() == api.HMM_EINVAL
    xy = obs.xy.copy()
    fl = obs.tremor.copy()
    fl[10] = 1
    xy[10, 0] = np.inf  # flagged tremor with a non-finite location
    assert math.isnan(_gpu_loglik(api, prm, xy, fl))
    assert ctx.hmm_status() == api.HMM_EINVAL


def test_host_argument_errors(cuda_lib):
    api = cuda_lib
    ctx = api.default_context()
    rng = np.random.default_rng(4)
    prm = synth.random_params(4, rng)
    t = api.to_device(prm)
    xy = torch.zeros(10, 2, device="cuda")
    fl = torch.zeros(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(api.HMMError) as e:
        ctx.hmm_loglik(*t, xy, fl, opts=api.make_opts(chunk_len=100))
    assert e.value.code == api.HMM_EINVAL
    with pytest.raises(api.HMMError):
        ctx.hmm_loglik_batched(t[0][None], t[1][None], t[2][None], t[3][None], t[4][None],
                               [0, 5, 3], xy, fl)


def test_batched_segments_fp32(cuda_lib):
    api = cuda_lib
    d = synth.batched_inputs(K=8, T=60_000, n_prop=6, seed=3, n_seg=7)
    ctx = api.default_context()
    pr = api.to_device(d["params"])
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    got = ctx.hmm_loglik_batched(*pr, d["offsets"], xy, fl, opts=api.make_opts(chunk_len=512))
    ref = oracle.loglik_batched(d["params"], d["xy"], d["tremor"], d["offsets"], n_threads=4)
    got = got.cpu().numpy()
    for q in range(6):
        assert _close(got[q], ref[q]), (q, got[q], ref[q])


def test_batched_empty_and_unit_segments(cuda_lib):
    api = cuda_lib
    rng = np.random.default_rng(8)
    gen = synth.random_params(5, rng)
    lens = [0, 1, 2, 700, 0, 65, 1]
    xy, fl, offs = synth.sample_segments(gen, lens, rng)
    props = synth.stack_params([synth.perturb_params(gen, rng) for _ in range(3)])
    ctx = api.default_context()
    got = ctx.hmm_loglik_batched(*api.to_device(props), offs, torch.from_numpy(xy).cuda(),
                                 torch.from_numpy(fl).cuda(), opts=api.make_opts(chunk_len=64))
    ref = oracle.loglik_batched(props, xy, fl, offs)
    got = got.cpu().numpy()
    for q in range(3):
        assert _close(got[q], ref[q]), (q, got[q], ref[q])


def test_host_entry_point_matches_device(cuda_lib):
    api = cuda_lib
    d = synth.batched_inputs(K=6, T=20_000, n_prop=4, seed=11, n_seg=3)
    ctx = api.default_context()
    dev = ctx.hmm_loglik_batched(*api.to_device(d["params"]), d["offsets"],
                                 torch.from_numpy(d["xy"]).cuda(), torch.from_numpy(d["tremor"]).cuda())
    host = ctx.hmm_loglik_batched_host(*d["params"].as_tuple(), d["offsets"], d["xy"], d["tremor"])
    assert np.array_equal(dev.cpu().numpy(), host)


def _split_favourites():
    """P = I, identical tremor locations for every state, p = (0.9, 0.001, 0.5,
    0.02), and T = 2049: tremors at steps 0..1024, none after. The first half
    favours the p = 0.9 state, the second the p = 0.001 state, and the whole
    the p = 0.5 state -- by 2^868 and 2^1022 behind the favourite of each
    half, far outside the float range."""
    rng = np.random.default_rng(2900)
    K = 4
    prm = synth.random_params(K, rng)
    prm.P[:] = np.eye(K, dtype=np.float32)
    prm.p_tremor[:] = np.array([0.9, 0.001, 0.5, 0.02], np.float32)
    prm.mu[:] = (150.0, 75.0)
    prm.cov[:] = (100.0, 0.0, 100.0)
    T = 2049
    fl = np.zeros(T, np.uint8)
    fl[:1025] = 1
    xy = np.where(fl[:, None] == 1, rng.normal((150.0, 75.0), 10.0, (T, 2)), 0.0).astype(np.float32)
    return prm, xy, fl


def test_reducible_transitions_tree(cuda_lib):
    # the product tree aligns every row of a product on its own scale: with
    # one alignment per matrix the p = 0.5 row of the second half's product
    # (2^1022 below its largest row) would flush, and with it the row that
    # carries the likelihood
    prm, xy, fl = _split_favourites()
    ref = oracle.loglik(prm, xy, fl)
    # closed form: log sum_k pi_k p_k^1025 (1 - p_k)^1024 + sum over tremors of log N(o_t)
    p = prm.p_tremor.astype(np.float64)
    terms = np.log(prm.pi.astype(np.float64)) + 1025 * np.log(p) + 1024 * np.log1p(-p)
    d = xy[:1025].astype(np.float64) - (150.0, 75.0)
    lgauss = -np.log(2 * np.pi * 100.0) - 0.5 * (d ** 2).sum(axis=1) / 100.0
    want = terms.max() + math.log(np.exp(terms - terms.max()).sum()) + lgauss.sum()
    assert abs(ref - want) < 1e-9 * abs(want), (ref, want)
    for L in (1024, 64):  # 2 and 32 chunks: one and two tree levels
        got = _gpu_loglik(cuda_lib, prm, xy, fl, chunk_len=L)
        assert _close(got, ref), (L, got, ref)
