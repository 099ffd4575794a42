"""Parity of the tensor-core (tcgen05) chunk products with the FP64 oracle.

Tolerance, per precision, an absolute bound in log L that grows with the
number of steps T (u: the operand's unit roundoff, 2^-11 for TF32, 2^-8 for
BF16):

* TF32-split (P carried as hi + lo, the running product rounded to nearest
  every step): |d| <= 8 sqrt(T) u. The per-step roundings are unbiased, so
  they add up like a random walk; P's own rounding error is O(u^2).
* TF32 (P rounded once): |d| <= 8 sqrt(T) u + T u / sqrt(K). Rounding P once
  changes every row sum of P by up to ~u / sqrt(K), a bias of that size per
  step. (The running product is truncated by the tensor core and the mean
  loss compensated in the emissions; what is left behaves like rounding.)
* BF16 (P as hi + lo, the running product in BF16): |d| <= 8 sqrt(T) u +
  4 T u^2, the second term an empirical allowance for the drift seen at long
  T (35 nats at T = 2^20, K = 32, both on the GPU and in a numpy replay of
  the kernels' rounding).

Full-size cases assert both this bound and the relative bar of the
tensor-core paths, |d| <= 1e-4 |log L|. Each test prints the observed error.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

TC_REL, TC_ABS = 1e-4, 1e-3
PRECS = ["tf32", "tf32_split", "bf16"]
UNIT = {"tf32": 2.0 ** -11, "tf32_split": 2.0 ** -11, "bf16": 2.0 ** -8}


def tol(prec, T, K):
    """Allowed |log L error| for a tensor-core precision on T observations, K states."""
    u = UNIT[prec]
    b = 8.0 * math.sqrt(max(T, 1)) * u
    if prec == "tf32":
        b += T * u / math.sqrt(K)
    elif prec == "bf16":
        b += 4.0 * T * u * u
    return b + TC_ABS


def check_full(prec, T, K, got, ref):
    """Both bounds at full size: the per-T absolute one and the relative bar."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    assert np.all(err <= tol(prec, T, K)), (prec, err.max(), tol(prec, T, K))
    assert np.all(err <= TC_REL * np.abs(ref)), (prec, (err / np.abs(ref)).max())


def _run(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    out = ctx.hmm_loglik(*api.to_device(prm), torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                         torch.from_numpy(np.ascontiguousarray(tremor)).cuda(), opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return float(out.item())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [1, 4, 16, 17, 25, 32, 33, 48, 49, 64, 65, 80])
def test_tc_parity_sizes(cuda_lib, K, prec):
    rng = np.random.default_rng(2000 + K)
    prm = synth.random_params(K, rng)
    T = 5000 + 37
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    for L in (64, 256, 0):
        got = _run(cuda_lib, prm, obs.xy, obs.tremor, precision=prec, chunk_len=L)
        err = abs(got - ref)
        print(f"K={K} {prec} L={L}: rel err {err / abs(ref):.2e}")
        assert err <= tol(prec, T, K), (K, prec, L, got, ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("T", [0, 1, 2, 65, 130])
def test_tc_small_T(cuda_lib, prec, T):
    rng = np.random.default_rng(300 + T)
    prm = synth.random_params(9, rng)
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    got = _run(cuda_lib, prm, obs.xy, obs.tremor, precision=prec, chunk_len=64)
    assert abs(got - ref) <= tol(prec, T, 9), (T, got, ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [64, 80])
@pytest.mark.parametrize("T", [0, 1, 2, 65, 130])
def test_tc_wide_small_T(cuda_lib, prec, K, T):
    rng = np.random.default_rng(700 + T + K)
    prm = synth.random_params(K, rng)
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    got = _run(cuda_lib, prm, obs.xy, obs.tremor, precision=prec, chunk_len=64)
    assert abs(got - ref) <= tol(prec, T, K), (K, T, got, ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [32, 48, 64, 80])
def test_tc_batched_segments(cuda_lib, prec, K):
    api = cuda_lib
    d = synth.batched_inputs(K=K, T=80_000, n_prop=12, seed=5, n_seg=7)
    ctx = api.default_context()
    got = ctx.hmm_loglik_batched(*api.to_device(d["params"]), d["offsets"],
                                 torch.from_numpy(d["xy"]).cuda(), torch.from_numpy(d["tremor"]).cuda(),
                                 opts=api.make_opts(precision=prec, chunk_len=256)).cpu().numpy()
    ref = oracle.loglik_batched(d["params"], d["xy"], d["tremor"], d["offsets"], n_threads=4)
    rel = np.abs(got - ref) / np.abs(ref)
    print(f"K={K} {prec} batched max rel err {rel.max():.2e}")
    Ts = np.diff(d["offsets"])
    for q in range(len(ref)):
        # per-segment bounds add up over the segments of one proposal
        bound = sum(tol(prec, int(t), K) for t in Ts)
        assert abs(got[q] - ref[q]) <= bound, (q, got[q] - ref[q], bound)
    assert np.all(rel <= TC_REL), rel


@pytest.mark.parametrize("prec", PRECS)
def test_tc_bit_reproducible(cuda_lib, prec):
    d = synth.config_inputs("k4_t1e4")
    a = _run(cuda_lib, d["params"], d["xy"], d["tremor"], precision=prec)
    b = _run(cuda_lib, d["params"], d["xy"], d["tremor"], precision=prec)
    assert a == b


def test_tc_zero_likelihood(cuda_lib):
    rng = np.random.default_rng(3)
    prm = synth.random_params(8, rng)
    prm.p_tremor[:] = 0.0
    xy = np.zeros((700, 2), np.float32)
    fl = np.zeros(700, np.uint8)
    fl[400] = 1
    assert _run(cuda_lib, prm, xy, fl, precision="tf32", chunk_len=64) == -math.inf


def test_tc_k25_t2p20(cuda_lib):
    d = synth.config_inputs("k25_t2p20")
    ref = oracle.loglik(d["params"], d["xy"], d["tremor"])
    for prec in PRECS:
        got = _run(cuda_lib, d["params"], d["xy"], d["tremor"], precision=prec)
        print(f"K=25 T=2^20 {prec}: rel err {abs(got - ref) / abs(ref):.2e}, abs {abs(got - ref):.3f}")
        check_full(prec, len(d["tremor"]), 25, got, ref)


def test_bench_workload_sampled(cuda_lib):
    """K=32, T=2^20, 256 proposals, automatic chunking (the benchmark's launch):
    every tensor-core precision against the oracle on sampled proposals, and
    against FP32-SIMT on all."""
    api = cuda_lib
    d = synth.batched_inputs(K=32, T=1 << 20, n_prop=256, seed=3)
    ctx = api.default_context()
    dev = api.to_device(d["params"])
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    fp = ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl, opts=api.make_opts(precision="fp32")).cpu().numpy()
    assert ctx.hmm_status() == api.HMM_OK
    tc = {}
    for prec in PRECS:
        tc[prec] = ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl,
                                          opts=api.make_opts(precision=prec)).cpu().numpy()
        assert ctx.hmm_status() == api.HMM_OK
        assert np.all(np.abs(tc[prec] - fp) <= TC_REL * np.abs(fp)), prec
    pick = [0, 77, 200, 255]
    sub = type(d["params"])(*(a[pick] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=4)
    print("sampled rel err fp32", np.abs(fp[pick] - ref) / np.abs(ref))
    assert np.all(np.abs(fp[pick] - ref) <= 1e-6 * np.abs(ref))
    for prec, v in tc.items():
        print(f"sampled rel err {prec}", np.abs(v[pick] - ref) / np.abs(ref))
        check_full(prec, 1 << 20, 32, v[pick], ref)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("K", [16, 32])
@pytest.mark.parametrize("R", [1, 3, 8])
def test_tc_renorm_intervals(cuda_lib, prec, K, R):
    """Renormalisation intervals other than the fast path's four (the general
    per-row path), ragged chunk tails included, against the oracle."""
    rng = np.random.default_rng(4100 + 10 * K + R)
    prm = synth.random_params(K, rng)
    T = 5000 + 37
    obs = synth.sample_observations(prm, T, rng)
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    got = _run(cuda_lib, prm, obs.xy, obs.tremor, precision=prec, chunk_len=256, renorm_every=R)
    assert abs(got - ref) <= tol(prec, T, K), (K, prec, R, got, ref)


@pytest.mark.parametrize("K", [64, 80])
def test_precision_sweep_wide_full_size(cuda_lib, K):
    """K=64 and K=80, T=2^22, 128 proposals (the precision-sweep workload):
    FP32-SIMT, TF32, TF32-split and BF16 chunk products on every proposal,
    the FP64 oracle on two sampled proposals; FP32 recheck agreement on all."""
    api = cuda_lib
    d = synth.batched_inputs(K=K, T=1 << 22, n_prop=128, seed=11)
    ctx = api.default_context()
    dev = api.to_device(d["params"])
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    res = {}
    for prec in ["fp32"] + PRECS:
        res[prec] = ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl,
                                           opts=api.make_opts(precision=prec)).cpu().numpy()
        assert ctx.hmm_status() == api.HMM_OK
    pick = [5, 100]
    sub = type(d["params"])(*(a[pick] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=2)
    for prec, v in res.items():
        rel = np.abs(v[pick] - ref) / np.abs(ref)
        print(f"K={K} T=2^22 {prec}: sampled rel err {rel.max():.2e}")
        if prec == "fp32":
            assert np.all(rel <= 1e-6), (prec, rel)
        else:
            check_full(prec, 1 << 22, K, v[pick], ref)
        if prec != "fp32":
            assert np.all(np.abs(v - res["fp32"]) <= TC_REL * np.abs(res["fp32"]))


def test_uneven_segments_full_size(cuda_lib):
    """K=32, 256 proposals, 64 segments of log-uniform length (1e3..1e6 steps,
    about 2^24 in total) shared by all proposals (the batched-MCMC workload):
    FP32-SIMT then TF32, both on every proposal; the FP64 oracle on two
    sampled proposals."""
    api = cuda_lib
    d = synth.batched_inputs(K=32, T=1 << 24, n_prop=256, seed=3, n_seg=64)
    assert len(d["offsets"]) == 65
    ctx = api.default_context()
    dev = api.to_device(d["params"])
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    fp = ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl, opts=api.make_opts(precision="fp32")).cpu().numpy()
    assert ctx.hmm_status() == api.HMM_OK
    tc = ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl, opts=api.make_opts(precision="tf32")).cpu().numpy()
    assert ctx.hmm_status() == api.HMM_OK
    assert np.all(np.abs(tc - fp) <= TC_REL * np.abs(fp))
    pick = [17, 230]
    sub = type(d["params"])(*(a[pick] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=2)
    print("64 segments, 2^24 steps: rel err fp32", np.abs(fp[pick] - ref) / np.abs(ref),
          "tf32", np.abs(tc[pick] - ref) / np.abs(ref))
    assert np.all(np.abs(fp[pick] - ref) <= 1e-6 * np.abs(ref))
    Ts = np.diff(d["offsets"])
    bound = sum(tol("tf32", int(t), 32) for t in Ts)
    assert np.all(np.abs(tc[pick] - ref) <= bound), (np.abs(tc[pick] - ref), bound)
    assert np.all(np.abs(tc[pick] - ref) <= TC_REL * np.abs(ref))
