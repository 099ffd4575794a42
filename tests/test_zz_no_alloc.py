"""The allocation-free entry point agrees with the context-based one.

hmm_loglik_noalloc exists for callers that cannot allocate device memory
during a call (frameworks that own every allocation, services with a fixed
device footprint, code that must not risk the synchronisation cudaMalloc can
cause). It keeps its scratch in one fixed __device__ array that every call
reuses, so this test makes two calls in a row with different inputs and
checks each against hmm_loglik (FP32-SIMT, the same chunk length), within
the FP32 tolerance the other parity tests use. It also checks that sizes
beyond the stated maximum are rejected.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""
import math

import numpy as np
import pytest
import torch

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


def test_noalloc_matches_context_path_twice(cuda_lib):
    api = cuda_lib
    cases = [(101, 25, 300_001), (202, 7, 4_000)]  # second call: smaller K and T
    for seed, K, T in cases:
        prm, obs = _inputs(seed, K, T)
        got = _noalloc(api, prm, obs)
        ref = _ref(api, prm, obs)
        assert math.isfinite(got)
        assert abs(got - ref) <= FP32_REL * abs(ref) + FP32_ABS, (K, T, got, ref)


def test_noalloc_largest_size_and_limits(cuda_lib):
    api = cuda_lib
    prm, obs = _inputs(303, 32, 1 << 20)
    got = _noalloc(api, prm, obs)
    ref = _ref(api, prm, obs)
    assert abs(got - ref) <= FP32_REL * abs(ref) + FP32_ABS, (got, ref)
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
