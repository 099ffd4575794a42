"""Replays the tensor-core kernels' rounding model in numpy at full size and
prints each precision's log-likelihood error against the FP64 oracle.

    python tests/replay_precision.py [n_proposals] [--sparse]   (about 5 minutes at 16)

Workload: the batched benchmark's inputs (K = 32, T = 2^20, proposals
0..n-1 of seed 3), or with --sparse its sparse-tremor workload (seed 103,
tremor probabilities in synth.SPARSE_P_RANGE). For every proposal the forward vector is advanced as the
kernels advance each row of a chunk product: the operand rounded every step
(TF32: half-ulp add on the bit pattern, low 13 bits cleared; BF16: round to
nearest even; or truncation), P rounded once as hi (+ lo), FP32 products
and emission scaling, exact power-of-two renormalisation. The errors it
prints can be set beside the errors measured on the GPU for the same
proposals (the benchmark's `error_vs_oracle`): where they agree, the kernels
compute exactly this model. Not collected by pytest (its name does not start
with test_); the rounding functions are those of test_precision_model.py.
"""
from __future__ import annotations

import math
import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
import tests.test_precision_model as pm  # noqa: E402
from paper_2003_03508_gb300 import synth  # noqa: E402


def replay(d, n, rnd_v, rnd_p, split, factor=1.0, block=4096):
    prm = d["params"]
    pi = prm.pi[:n].astype(np.float64)
    P = prm.P[:n].astype(np.float32)
    p = prm.p_tremor[:n].astype(np.float64)
    mu = prm.mu[:n].astype(np.float64)
    cov = prm.cov[:n].astype(np.float64)
    det = cov[:, :, 0] * cov[:, :, 2] - cov[:, :, 1] ** 2
    ia, ib, ic = cov[:, :, 2] / det, -cov[:, :, 1] / det, cov[:, :, 0] / det
    lno = np.log1p(-p)
    ltr = np.log(p) - np.log(2 * np.pi) - 0.5 * np.log(det)
    xy = d["xy"].astype(np.float64)
    fl = d["tremor"]
    T = xy.shape[0]
    Ph = rnd_p(P).astype(np.float64)
    Pl = rnd_p(P - rnd_p(P)).astype(np.float64) if split else None
    v = pi.copy()
    logL = np.zeros(n)
    for b0 in range(0, T, block):
        x = xy[b0:b0 + block]
        dx = x[:, None, None, 0] - mu[None, :, :, 0]
        dy = x[:, None, None, 1] - mu[None, :, :, 1]
        q = ia[None] * dx * dx + 2 * ib[None] * dx * dy + ic[None] * dy * dy
        le = np.where(fl[b0:b0 + block, None, None] == 1, ltr[None] - 0.5 * q, lno[None])
        for j in range(le.shape[0]):
            if b0 + j > 0:
                a = rnd_v(v.astype(np.float32)).astype(np.float64)
                w = np.einsum("pk,pkj->pj", a, Ph)
                if split:
                    w += np.einsum("pk,pkj->pj", a, Pl)
                v = w.astype(np.float32).astype(np.float64)
            m = le[j].max(axis=1)
            dd = (np.exp(le[j] - m[:, None]) * factor).astype(np.float32)
            v = (v * dd).astype(np.float32).astype(np.float64)
            e = np.frexp(v.sum(axis=1))[1]
            v = v * np.ldexp(1.0, -e)[:, None]
            logL += m + e * math.log(2.0)
    return logL + np.log(v.sum(axis=1))


def main(n=16, sparse=False):
    if sparse:
        d = synth.batched_inputs(K=32, T=1 << 20, n_prop=max(n, 1), seed=103, sparse=True)
    else:
        d = synth.batched_inputs(K=32, T=1 << 20, n_prop=max(n, 1), seed=3)
    sub = type(d["params"])(*(a[:n] for a in d["params"].as_tuple()))
    ref = oracle.loglik_batched(sub, d["xy"], d["tremor"], d["offsets"], n_threads=8)
    f = 1.0 / (1.0 - pm.TRUNC_MEAN_LOSS)
    cases = (("tf32", (pm.rna_tf32, pm.rna_tf32, False)),
             ("tf32_split", (pm.rna_tf32, pm.rna_tf32, True)),
             ("bf16 (hi+lo P)", (pm.rne_bf16, pm.rne_bf16, True)),
             ("tf32 truncated + compensation", (pm.trunc_tf32, pm.rna_tf32, False, f)),
             ("tf32_split truncated + compensation", (pm.trunc_tf32, pm.rna_tf32, True, f)))
    for name, args in cases:
        t0 = time.time()
        err = replay(d, n, *args) - ref
        rel = np.abs(err) / np.abs(ref)
        print(f"{name}: max |err| {np.abs(err).max():.2f} nats, max rel {rel.max():.2e}, "
              f"mean err {err.mean():+.2f} ({time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    main(int(args[0]) if args else 16, sparse="--sparse" in sys.argv)
