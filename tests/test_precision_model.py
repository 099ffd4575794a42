"""The error model behind the tensor-core tolerances, checked by emulation.

The tensor-core chunk kernels reduce the running product to the operand type
at every step and hold P as one rounded image (TF32) or as hi + lo images
(TF32-split, BF16): TF32-split and BF16 round each operand to nearest, and
plain TF32 hands the raw FP32 bits to the tensor core, which truncates them,
with the mean loss compensated in the emission factors (the last bullet
below). This test replays that arithmetic in numpy on the
forward vector -- FP32 products and emission scaling, operands rounded
exactly as the kernels round them (TF32: half-ulp add on the bit pattern,
the low 13 bits cleared; BF16: round to nearest even), exact power-of-two
renormalisation -- and compares log L with the FP64 oracle. It pins the
readings the GPU tolerances rest on:

* rounding the operand every step costs O(sqrt(T) u) in log L: TF32-split
  and BF16 hi+lo stay within the per-T bound 8 sqrt(T) u;
* rounding P once (plain TF32) adds a bias that grows like T u, which the
  1e-4 relative tolerance absorbs on tremor-shaped data;
* without the hi + lo split, BF16's rounding of P drifts past the tolerance
  (the reason P is carried as hi + lo);
* truncating to TF32 instead of rounding (what the tensor core does to the
  low bits it ignores) biases every step and also leaves the tolerance;
* but that bias is a known mean: with mantissas spread log-uniformly over
  [1, 2) (as in long products of random factors), truncating 13 bits loses
  on average c = 2^-11 (1 - 1/2) / ln 2 of the value, so multiplying each
  step's emission factors by 1 / (1 - c) -- free, as they are computed once
  per step -- leaves an error as small as rounding's, on tremor-shaped and
  on sparse-tremor data (the reading the plain TF32 kernels use: they no
  longer round each element in the epilogue).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2003_03508_gb300 import synth


def rna_tf32(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x1000) & 0xFFFFE000).astype(np.uint32).view(np.float32)


def trunc_tf32(x):
    return (np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def rne_bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


U = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -9}


def _case(K, T, seed):
    rng = np.random.default_rng(seed)
    prm = synth.random_params(K, rng)
    obs = synth.sample_observations(prm, T, rng)
    le = np.array([oracle.log_emission(prm, float(obs.xy[t, 0]), float(obs.xy[t, 1]), int(obs.tremor[t]))
                   for t in range(T)])
    return prm, obs, le, oracle.loglik(prm, obs.xy, obs.tremor)


def _emulate(prm, le, rnd, split, rnd_p=None, factor=1.0):
    """log L with the kernels' operand rounding (emit-first): the running
    vector is rounded by `rnd` every step, P once by `rnd_p` (default `rnd`),
    as hi (+ lo with split); every step's emission factors are multiplied by
    `factor` (which is not divided out again)."""
    rnd_p = rnd_p or rnd
    P = prm.P.astype(np.float32)
    Ph = rnd_p(P).astype(np.float64)
    Pl = rnd_p(P - rnd_p(P)).astype(np.float64) if split else None
    v = prm.pi.astype(np.float64)
    logL = 0.0
    for t in range(le.shape[0]):
        if t > 0:
            a = rnd(v.astype(np.float32)).astype(np.float64)
            w = a @ Ph
            if split:
                w = w + a @ Pl
            v = w.astype(np.float32).astype(np.float64)          # FP32 accumulator
        m = le[t].max()
        d = (np.exp(le[t] - m) * factor).astype(np.float32)      # emission factors in FP32
        v = (v * d).astype(np.float32).astype(np.float64)
        e = math.frexp(v.sum())[1]
        v = v * 2.0 ** (-e)                                      # exact power-of-two renorm
        logL += m + e * math.log(2.0)
    return logL + math.log(v.sum())


def _tol(u, T, ref):
    """The GPU tests' tolerance: max(1e-4 |log L|, 8 sqrt(T) u) + 1e-3."""
    return max(1e-4 * abs(ref), 8.0 * math.sqrt(T) * u) + 1e-3


@pytest.fixture(scope="module")
def long_case():
    return _case(8, 20_000, 2)


@pytest.mark.parametrize("T,seed", [(3000, 1), (20_000, 2)])
def test_split_precisions_stay_within_the_sqrt_T_bound(T, seed, long_case):
    prm, obs, le, ref = long_case if T == 20_000 else _case(8, T, seed)
    for rnd, u in ((rna_tf32, U["tf32"]), (rne_bf16, U["bf16"])):
        err = abs(_emulate(prm, le, rnd, split=True) - ref)
        assert err <= 8.0 * math.sqrt(T) * u, (rnd.__name__, err)


def test_single_rounded_P_is_a_bias_the_relative_tolerance_absorbs(long_case):
    prm, obs, le, ref = long_case
    T = le.shape[0]
    err = abs(_emulate(prm, le, rna_tf32, split=False) - ref)
    assert err <= _tol(U["tf32"], T, ref)
    # larger than the split's error: the bias of rounding P once
    assert err > 4 * abs(_emulate(prm, le, rna_tf32, split=True) - ref)


def test_bf16_needs_the_split(long_case):
    prm, obs, le, ref = long_case
    T = le.shape[0]
    assert abs(_emulate(prm, le, rne_bf16, split=False) - ref) > _tol(U["bf16"], T, ref)


def test_truncation_instead_of_rounding_fails(long_case):
    prm, obs, le, ref = long_case
    T = le.shape[0]
    err = _emulate(prm, le, trunc_tf32, split=False) - ref
    assert err < 0 and abs(err) > _tol(U["tf32"], T, ref)


TRUNC_MEAN_LOSS = 2.0 ** -11 * 0.5 / math.log(2.0)


def _sparse_case(K, T, seed):
    rng = np.random.default_rng(seed)
    prm = synth.random_params(K, rng, p_range=synth.SPARSE_P_RANGE)
    obs = synth.sample_observations(prm, T, rng)
    le = np.array([oracle.log_emission(prm, float(obs.xy[t, 0]), float(obs.xy[t, 1]), int(obs.tremor[t]))
                   for t in range(T)])
    return prm, obs, le, oracle.loglik(prm, obs.xy, obs.tremor)


@pytest.mark.parametrize("which", ["standard", "sparse"])
def test_truncation_with_mean_loss_compensation(which, long_case):
    prm, obs, le, ref = long_case if which == "standard" else _sparse_case(8, 20_000, 4)
    T = le.shape[0]
    f = 1.0 / (1.0 - TRUNC_MEAN_LOSS)
    plain = abs(_emulate(prm, le, trunc_tf32, split=True, rnd_p=rna_tf32) - ref)
    comp = abs(_emulate(prm, le, trunc_tf32, split=True, rnd_p=rna_tf32, factor=f) - ref)
    # the compensation removes the truncation bias: within the sqrt(T) bound,
    # and within 0.1 nats of what rounding gives with P rounded once
    assert comp <= 8.0 * math.sqrt(T) * U["tf32"] and comp < plain / 10, (comp, plain)
    rna1 = _emulate(prm, le, rna_tf32, split=False) - ref
    comp1 = _emulate(prm, le, trunc_tf32, split=False, rnd_p=rna_tf32, factor=f) - ref
    assert abs(comp1 - rna1) < 0.1, (comp1, rna1)
