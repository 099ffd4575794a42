"""The chunk-length tuner on the GPU: it measures its candidates, stores the
fastest, later automatic calls use it, and the tuned results match the FP64
oracle at the precision's tolerance (FP32 1e-6, tensor cores 1e-4 relative
in log L).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu

REL = {"fp32": 1e-6, "tf32": 1e-4}


@pytest.mark.parametrize("prec", ["fp32", "tf32"])
def test_autotune_stores_and_reuses_the_fastest(cuda_lib, prec):
    api = cuda_lib
    d = synth.batched_inputs(K=8, T=40_000, n_prop=6, seed=11, n_seg=3)
    dev = api.to_device(d["params"])
    xy, fl = torch.from_numpy(d["xy"]).cuda(), torch.from_numpy(d["tremor"]).cuda()
    offs = d["offsets"]
    n_seg, steps = len(offs) - 1, api.chain_steps(offs)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ctx = api.Context(0)
    api.tune_clear()
    try:
        out, L, ms = ctx.hmm_autotune_batched(*dev, offs, xy, fl, opts=api.make_opts(precision=prec), reps=2)
        assert L in api.tune_candidates(prec, 6, 8, steps, sms)
        assert ms > 0.0
        assert ctx.last_chunk_len == L
        assert api.tune_lookup(sms, 8, prec, 6, n_seg, steps) == L
        ref = oracle.loglik_batched(d["params"], d["xy"], d["tremor"], offs, n_threads=4)
        got = out.cpu().numpy()
        rel = np.abs(got - ref) / np.abs(ref)
        print(f"{prec}: tuned L={L} ({ms:.3f} ms), max rel err {rel.max():.2e}")
        assert np.all(rel <= REL[prec]), rel
        # an automatic call now uses the tuned length, and gives the same bits
        again = ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=api.make_opts(precision=prec))
        assert ctx.last_chunk_len == L
        assert torch.equal(again, out)
        # without the entry the cost model decides again
        api.tune_clear()
        ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=api.make_opts(precision=prec))
        assert ctx.last_chunk_len == api.default_chunk_len(prec, 6, 8, steps, sms)
        # a fixed chunk length cannot be tuned
        with pytest.raises(api.HMMError) as e:
            ctx.hmm_autotune_batched(*dev, offs, xy, fl, opts=api.make_opts(precision=prec, chunk_len=256))
        assert e.value.code == api.HMM_EINVAL
        assert ctx.hmm_status() == api.HMM_OK
    finally:
        api.tune_clear()
        ctx.close()
