"""Posterior state probabilities on the GPU (hmm_posterior) against the FP64
forward-backward oracle.

Tolerance: |gamma_gpu - gamma_oracle| <= 2e-4 per entry (probabilities in
[0, 1]). The error budget: the forward and backward vectors are carried in
FP32 and renormalised every step (relative error ~1e-7 per step, the
normalised recursion contracts it), the chunk products enter through the
boundary vectors, and the per-step posterior is a normalised product of the
two. The most probable state per step must agree wherever the oracle's top
two probabilities differ by more than the tolerance.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 2e-4


def _run(api, prm, obs, **opt):
    ctx = api.default_context()
    g, ll = ctx.hmm_posterior(*api.to_device(prm), torch.from_numpy(np.ascontiguousarray(obs.xy)).cuda(),
                              torch.from_numpy(np.ascontiguousarray(obs.tremor)).cuda(),
                              opts=api.make_opts(**opt))
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.float64), float(ll.item())


def _check(g, ref, tol=TOL):
    err = np.abs(g - ref).max()
    assert err <= tol, err
    top2 = np.sort(ref, axis=1)[:, -2:]
    clear = (top2[:, 1] - top2[:, 0]) > 2 * tol
    assert np.array_equal(g.argmax(1)[clear], ref.argmax(1)[clear])
    return err


@pytest.mark.parametrize("K", [2, 3, 7, 16, 25, 32, 33, 64, 80])
def test_posterior_parity_sizes(cuda_lib, K):
    rng = np.random.default_rng(900 + K)
    prm = synth.random_params(K, rng)
    T = 4000 + 17
    obs = synth.sample_observations(prm, T, rng)
    ref, rll = oracle.posterior(prm, obs.xy, obs.tremor)
    for L in (64, 512):
        g, ll = _run(cuda_lib, prm, obs, chunk_len=L)
        err = _check(g, ref)
        print(f"K={K} L={L}: max |gamma err| {err:.2e}")
        assert abs(ll - rll) <= 1e-6 * abs(rll)


@pytest.mark.parametrize("T", [1, 2, 3, 64, 65, 66, 130])
@pytest.mark.parametrize("init_mode", [0, 1])
def test_posterior_small_T(cuda_lib, T, init_mode):
    rng = np.random.default_rng(950 + T)
    prm = synth.random_params(5, rng)
    obs = synth.sample_observations(prm, T, rng)
    ref, _ = oracle.posterior(prm, obs.xy, obs.tremor, init_mode)
    g, _ = _run(cuda_lib, prm, obs, chunk_len=64, init_mode=init_mode)
    _check(g, ref)


@pytest.mark.parametrize("prec,tol", [("tf32", 1e-3), ("tf32_split", 1e-3), ("bf16", 2e-2)])
def test_posterior_tensor_core_products(cuda_lib, prec, tol):
    """With tensor-core chunk products the boundary vectors carry the
    products' operand rounding (relative ~sqrt(L) u per chunk, u = 2^-11 for
    TF32, 2^-9 for BF16), so the posterior's error grows accordingly; the
    within-chunk recursions stay FP32."""
    rng = np.random.default_rng(77)
    prm = synth.random_params(32, rng)
    obs = synth.sample_observations(prm, 20000, rng)
    ref, _ = oracle.posterior(prm, obs.xy, obs.tremor)
    g, _ = _run(cuda_lib, prm, obs, precision=prec, chunk_len=512)
    print(prec, "max |gamma err|", np.abs(g - ref).max())
    _check(g, ref, tol=tol)


def test_posterior_long_sequence(cuda_lib):
    """K=25 (24 spatial states and a quiescent one), T=2^20: every step against the oracle."""
    d = synth.config_inputs("k25_t2p20")
    ref, rll = oracle.posterior(d["params"], d["xy"], d["tremor"])
    g, ll = _run(cuda_lib, d["params"], type("O", (), {"xy": d["xy"], "tremor": d["tremor"]}))
    err = _check(g, ref)
    print("K=25 T=2^20 max |gamma err|", err)
    assert np.all(np.abs(g.sum(1) - 1) < 1e-4)
    assert abs(ll - rll) <= 1e-6 * abs(rll)
