"""The allocation-free entry point against the FP64 oracle and the context path.

hmm_loglik_noalloc exists for callers that cannot allocate device memory
during a call (frameworks that own every allocation, services with a fixed
device footprint, code that must not risk the synchronisation cudaMalloc can
cause). It keeps its scratch in one fixed __device__ array that every call
reuses, so this test makes two calls in a row with different inputs and
checks each against the FP64 CPU oracle and against hmm_loglik (FP32-SIMT,
the same chunk length), within the FP32 tolerance the other parity tests
use. It also checks that sizes beyond the stated maximum are rejected, that a
device-side failure (an observation far outside the representable range)
comes back as a NaN result because there is no context to report it through,
and that repeated calls leave the device's free memory unchanged.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_REL, FP32_ABS = 1e-6, 1e-4


def _inputs(seed, K, T):
    rng = np.random.default_rng(seed)
    prm = synth.random_params(K, rng)
    obs = synth.sample_observations(prm, T, rng)
    return prm, obs


def _ref(api, prm, obs):
    ctx = api.default_context()
    dev = api.to_device(prm)
    out = ctx.hmm_loglik(*dev, torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda(),
                         opts=api.make_opts(precision="fp32", chunk_len=1024))
    torch.cuda.synchronize()
    return float(out.item())


def _noalloc(api, prm, obs):
    dev = api.to_device(prm)
    out = api.hmm_loglik_noalloc(*dev, torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda())
    torch.cuda.synchronize()
    return float(out.item())


def test_noalloc_matches_oracle_and_context_path_twice(cuda_lib):
    api = cuda_lib
    cases = [(101, 25, 300_001), (202, 7, 4_000)]  # second call: smaller K and T
    for seed, K, T in cases:
        prm, obs = _inputs(seed, K, T)
        got = _noalloc(api, prm, obs)
        want = oracle.loglik(prm, obs.xy, obs.tremor)
        assert math.isfinite(got)
        assert abs(got - want) <= FP32_REL * abs(want) + FP32_ABS, (K, T, got, want)
        ref = _ref(api, prm, obs)
        assert abs(got - ref) <= FP32_REL * abs(ref) + FP32_ABS, (K, T, got, ref)


def test_noalloc_largest_size_and_limits(cuda_lib):
    api = cuda_lib
    prm, obs = _inputs(303, 32, 1 << 20)
    got = _noalloc(api, prm, obs)
    want = oracle.loglik(prm, obs.xy, obs.tremor)
    assert abs(got - want) <= FP32_REL * abs(want) + FP32_ABS, (got, want)
    # beyond the maximum: rejected, nothing computed
    prm33, obs33 = _inputs(304, 33, 100)
    with pytest.raises(api.HMMError) as e:
        _noalloc(api, prm33, obs33)
    assert e.value.code == api.HMM_EINVAL
    long_obs = synth.Observations(np.zeros(((1 << 20) + 1, 2), np.float32),
                                  np.zeros((1 << 20) + 1, np.uint8))
    with pytest.raises(api.HMMError) as e:
        _noalloc(api, prm, long_obs)
    assert e.value.code == api.HMM_EINVAL


def test_noalloc_reports_a_device_failure_as_nan(cuda_lib):
    """A tremor 10^6 km from every state puts the step's best emission below
    2^-65536 (out of range); the context path reports HMM_ENUMERIC through
    hmm_status, the allocation-free call returns NaN. The next, valid call
    is unaffected (the status word is cleared at the start of every call)."""
    api = cuda_lib
    prm, obs = _inputs(405, 6, 5000)
    xy = obs.xy.copy()
    fl = obs.tremor.copy()
    xy[2500] = (1e6, 1e6)
    fl[2500] = 1
    got = _noalloc(api, prm, synth.Observations(xy, fl))
    assert math.isnan(got), got
    ctx = api.Context()
    dev = api.to_device(prm)
    ctx.hmm_loglik(*dev, torch.from_numpy(xy).cuda(), torch.from_numpy(fl).cuda(),
                   opts=api.make_opts(precision="fp32", chunk_len=1024))
    assert ctx.hmm_status() == api.HMM_ENUMERIC
    ctx.close()
    got2 = _noalloc(api, prm, obs)
    want = oracle.loglik(prm, obs.xy, obs.tremor)
    assert abs(got2 - want) <= FP32_REL * abs(want) + FP32_ABS, (got2, want)


def test_noalloc_leaves_free_device_memory_unchanged(cuda_lib):
    """Ten calls after a warm-up call: the device's free memory (as the
    driver reports it) is the same before and after, so no call keeps an
    allocation; every input and output tensor exists before the first
    measurement."""
    api = cuda_lib
    prm, obs = _inputs(506, 16, 50_000)
    dev = api.to_device(prm)
    xy = torch.from_numpy(obs.xy).cuda()
    fl = torch.from_numpy(obs.tremor).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    api.hmm_loglik_noalloc(*dev, xy, fl, out=out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    vals = []
    for _ in range(10):
        api.hmm_loglik_noalloc(*dev, xy, fl, out=out)
        torch.cuda.synchronize()
        vals.append(float(out.item()))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert len(set(vals)) == 1  # same inputs, same scratch reuse: bit-for-bit repeatable
