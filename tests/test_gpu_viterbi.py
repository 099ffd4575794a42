"""The Viterbi path on the GPU (hmm_viterbi) against the FP64 oracle.

What is unique is the best score: the GPU's path, scored by the oracle in
FP64, must reach the oracle's maximum within 1e-7 relative (FP32 scores
within chunks can break near-ties differently), its reported score must be
its path's score within the same bound, and the two paths must agree on at
least 99.9% of the steps (they differ only around near-ties).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu
REL = 1e-7


def _run(api, prm, xy, tremor, **opt):
    ctx = api.default_context()
    path, score, ll = ctx.hmm_viterbi(*api.to_device(prm), torch.from_numpy(np.ascontiguousarray(xy)).cuda(),
                                      torch.from_numpy(np.ascontiguousarray(tremor)).cuda(),
                                      opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return path.cpu().numpy(), float(score.item()), float(ll.item())


def _check(prm, xy, tremor, path, score, mode=0):
    ref_path, ref = oracle.viterbi(prm, xy, tremor, mode)
    got = oracle.path_logjoint(prm, xy, tremor, path, mode)
    tol = REL * abs(ref) + 1e-9
    assert got >= ref - tol, (got, ref)
    assert abs(score - got) <= tol + 1e-6, (score, got)
    agree = float(np.mean(path == ref_path))
    assert agree >= 0.999, agree
    return agree


@pytest.mark.parametrize("K", [2, 3, 7, 16, 25, 32, 33, 64, 80])
def test_viterbi_parity_sizes(cuda_lib, K):
    rng = np.random.default_rng(1500 + K)
    prm = synth.random_params(K, rng)
    obs = synth.sample_observations(prm, 4000 + 21, rng)
    for L in (64, 0):
        path, score, ll = _run(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=L)
        a = _check(prm, obs.xy, obs.tremor, path, score)
        print(f"K={K} L={L}: path agreement {a:.5f}")
        assert score <= ll


@pytest.mark.parametrize("T", [1, 2, 3, 64, 65, 130])
@pytest.mark.parametrize("mode", [0, 1])
def test_viterbi_small_T(cuda_lib, T, mode):
    rng = np.random.default_rng(1600 + T)
    prm = synth.random_params(4, rng)
    obs = synth.sample_observations(prm, T, rng)
    path, score, _ = _run(cuda_lib, prm, obs.xy, obs.tremor, chunk_len=64, init_mode=mode)
    _check(prm, obs.xy, obs.tremor, path, score, mode)


def test_viterbi_long_sequence(cuda_lib):
    """K=25 (24 spatial states and a quiescent one), T=2^20."""
    d = synth.config_inputs("k25_t2p20")
    path, score, ll = _run(cuda_lib, d["params"], d["xy"], d["tremor"])
    a = _check(d["params"], d["xy"], d["tremor"], path, score)
    print("K=25 T=2^20 path agreement", a)
