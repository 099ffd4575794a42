"""Graph replay of the batched likelihood call.

A repeated hmm_loglik_batched call (same shape, offsets, options, pointers
and workspace) is captured into a CUDA graph on its second occurrence and
replayed from the third on. These tests check that the replayed graph gives
bit-for-bit the results of direct launches, that it reads the inputs'
current contents (new values in the same tensors give the new likelihood,
checked against the FP64 oracle), that any change of pointer, option or
segment layout goes back to direct launches, and that phase profiling and a
caller's own stream capture keep launching directly.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

FP32_REL = 1e-6


def _setup(api, seed=21, K=12, n_prop=6, T=20_000, n_seg=3):
    d = synth.batched_inputs(K=K, T=T, n_prop=n_prop, seed=seed, n_seg=n_seg)
    dev = [t.contiguous() for t in api.to_device(d["params"])]
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    out = torch.empty(n_prop, dtype=torch.float64, device="cuda")
    return d, dev, xy, fl, out


def _call(ctx, api, dev, offsets, xy, fl, out, **opt):
    ctx.hmm_loglik_batched(*dev, offsets, xy, fl, opts=api.make_opts(**opt), out=out)
    torch.cuda.synchronize()
    return out.cpu().numpy().copy(), ctx.last_call_graph


def test_replay_matches_direct_launches(cuda_lib):
    api = cuda_lib
    d, dev, xy, fl, out = _setup(api)
    ctx = api.Context()
    try:
        for prec in ("fp32", "tf32"):
            modes, vals = [], []
            for _ in range(4):
                v, m = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision=prec)
                vals.append(v)
                modes.append(m)
            assert modes == [0, 1, 2, 2], (prec, modes)
            ctx.set_call_graphs(False)
            direct, m = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision=prec)
            assert m == 0
            ctx.set_call_graphs(True)
            for v in vals:
                assert np.array_equal(v, direct), prec
            assert ctx.hmm_status() == api.HMM_OK
    finally:
        ctx.close()


def test_replay_reads_current_inputs(cuda_lib):
    """New parameter and observation values written into the same tensors:
    the replayed graph computes the new likelihood (FP64 oracle)."""
    api = cuda_lib
    d, dev, xy, fl, out = _setup(api, seed=22)
    ctx = api.Context()
    try:
        for _ in range(3):
            _call(ctx, api, dev, d["offsets"], xy, fl, out, precision="fp32")
        # other parameter sets (same K and count) and every tremor moved by 3 km
        prm2 = synth.batched_inputs(K=12, T=1000, n_prop=6, seed=23)["params"]
        xy2 = (d["xy"] + np.float32(3.0)).astype(np.float32)
        for t, a in zip(dev, api.to_device(prm2)):
            t.copy_(a)
        xy.copy_(torch.from_numpy(xy2))
        got, m = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision="fp32")
        assert m == 2
        ref = oracle.loglik_batched(prm2, xy2, d["tremor"], d["offsets"], n_threads=4)
        old = oracle.loglik_batched(d["params"], d["xy"], d["tremor"], d["offsets"], n_threads=4)
        assert np.all(np.abs(ref - old) > 1.0)  # the change is visible in every result
        assert np.all(np.abs(got - ref) <= FP32_REL * np.abs(ref)), np.abs(got - ref) / np.abs(ref)
    finally:
        ctx.close()


def test_changes_go_back_to_direct_launches(cuda_lib):
    api = cuda_lib
    d, dev, xy, fl, out = _setup(api, seed=24)
    ctx = api.Context()
    try:
        base = None
        for _ in range(3):
            base, m = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision="tf32")
        assert m == 2
        # another output tensor: a new configuration
        out2 = torch.empty_like(out)
        v, m = _call(ctx, api, dev, d["offsets"], xy, fl, out2, precision="tf32")
        assert m == 0 and np.array_equal(v, base)
        # another option
        v, m = _call(ctx, api, dev, d["offsets"], xy, fl, out2, precision="tf32", chunk_len=128)
        assert m == 0
        # other segment offsets (same total): the plan changes
        offs = d["offsets"].copy()
        offs[1] += 7
        v, m = _call(ctx, api, dev, offs, xy, fl, out2, precision="tf32")
        assert m == 0
        v2, m = _call(ctx, api, dev, offs, xy, fl, out2, precision="tf32")
        assert m == 1 and np.array_equal(v, v2)
        # profiling on: direct launches, same values
        ctx.hmm_profile_enable(True)
        v3, m = _call(ctx, api, dev, offs, xy, fl, out2, precision="tf32")
        assert m == 0 and np.array_equal(v, v3)
        ctx.hmm_profile_enable(False)
    finally:
        ctx.close()


def test_call_inside_a_caller_capture_launches_directly(cuda_lib):
    """A caller that captures its own stream gets the kernels in its graph."""
    api = cuda_lib
    d, dev, xy, fl, out = _setup(api, seed=25)
    ctx = api.Context()
    try:
        ref, _ = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision="fp32")  # plan and workspace
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        out.zero_()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s, capture_error_mode="relaxed"):
            ctx.hmm_loglik_batched(*dev, d["offsets"], xy, fl, opts=api.make_opts(precision="fp32"), out=out,
                                   stream=s)
        assert ctx.last_call_graph == 0
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        ctx.close()


def test_host_and_single_sequence_entry_points_replay(cuda_lib):
    """The host-buffer entry point (copies into the context's own device
    buffers, so its calls repeat even with fresh host arrays) and the
    single-sequence call replay too, with the direct launches' results."""
    api = cuda_lib
    d, dev, xy, fl, out = _setup(api, seed=26)
    ctx = api.Context()
    try:
        direct, _ = _call(ctx, api, dev, d["offsets"], xy, fl, out, precision="tf32")
        host_args = [np.asarray(a, np.float32) for a in d["params"].as_tuple()]
        modes = []
        for _ in range(3):
            v = ctx.hmm_loglik_batched_host(*host_args, d["offsets"], d["xy"], d["tremor"],
                                            opts=api.make_opts(precision="tf32"))
            modes.append(ctx.last_call_graph)
            assert np.array_equal(v, direct)
        assert modes == [0, 1, 2], modes
        # one sequence, one parameter set
        prm = synth.random_params(9, np.random.default_rng(27))
        obs = synth.sample_observations(prm, 7000, np.random.default_rng(28))
        one = api.to_device(prm)
        oxy = torch.from_numpy(obs.xy).cuda()
        ofl = torch.from_numpy(obs.tremor).cuda()
        res = torch.empty(1, dtype=torch.float64, device="cuda")
        modes, vals = [], []
        for _ in range(3):
            ctx.hmm_loglik(*one, oxy, ofl, opts=api.make_opts(precision="fp32"), out=res)
            torch.cuda.synchronize()
            modes.append(ctx.last_call_graph)
            vals.append(float(res.item()))
        assert modes == [0, 1, 2], modes
        assert len(set(vals)) == 1
        ref = oracle.loglik(prm, obs.xy, obs.tremor)
        assert abs(vals[0] - ref) <= FP32_REL * abs(ref), (vals[0], ref)
    finally:
        ctx.close()
