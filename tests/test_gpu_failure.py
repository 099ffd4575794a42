"""Failure detection on the device: a bounded wait that runs out.

Every tensor-core kernel waits on its mbarriers with a bounded wait that, when
it runs out, raises ETIMEOUT in the status word, sets the CTA's abort flag and
returns. hmm_check_bounded_wait runs that wait on a barrier phase that nothing
completes (a flag nothing sets), with a short limit: the call must come back
with HMM_ETIMEOUT after about the limit, and the context must stay usable (a
likelihood evaluation right after it matches the oracle).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2003_03508_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports(cuda_lib):
    api = cuda_lib
    for limit in (5.0, 20.0):
        rc, waited = api.check_bounded_wait(limit, torch.cuda.current_device())
        assert rc == api.HMM_ETIMEOUT, rc
        # measured in cycles at the rated clock; the SM may run slower or faster
        assert 0.4 * limit <= waited <= 3.0 * limit, (limit, waited)
    rng = np.random.default_rng(8)
    prm = synth.random_params(6, rng)
    obs = synth.sample_observations(prm, 3000, rng)
    ctx = api.Context()
    got = ctx.hmm_loglik(*api.to_device(prm), torch.from_numpy(obs.xy).cuda(), torch.from_numpy(obs.tremor).cuda(),
                         opts=api.make_opts(precision="tf32", chunk_len=256))
    assert ctx.hmm_status() == api.HMM_OK
    ref = oracle.loglik(prm, obs.xy, obs.tremor)
    assert abs(float(got.item()) - ref) <= 1e-4 * abs(ref)
    ctx.close()


def test_bounded_wait_rejects_bad_limits(cuda_lib):
    api = cuda_lib
    assert api.check_bounded_wait(0.0)[0] == api.HMM_EINVAL
    assert api.check_bounded_wait(1e6)[0] == api.HMM_EINVAL
