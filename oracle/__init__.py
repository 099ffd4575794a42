"""CPU oracle for the tremor-HMM likelihood -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The product path (the CUDA library and
its binding) never does, and the two share no code.

The C source (``hmm_oracle.c``) is compiled with plain ``gcc -O2`` (no fast
math) into ``_build/liboracle.so`` on first use, or by ``build()``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = [_HERE / "hmm_oracle.c", _HERE / "mcmc_oracle.c", _HERE / "mlp_oracle.c", _HERE / "twalk_oracle.c"]
_BUILD = _HERE / "_build"
_lib = None


def _digest() -> str:
    h = hashlib.sha1()
    for s in _SRC:
        if s.exists():
            h.update(s.read_bytes())
    return h.hexdigest()[:12]


def build(force: bool = False) -> Path:
    """Compile the oracle into a shared library (idempotent, keyed by source hash)."""
    _BUILD.mkdir(exist_ok=True)
    so = _BUILD / f"liboracle_{_digest()}.so"
    if so.exists() and not force:
        return so
    srcs = [str(s) for s in _SRC if s.exists()]
    tmp = so.with_suffix(f".tmp{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-o", str(tmp), *srcs, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, so)
    return so


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(str(build()))
        _declare(_lib)
    return _lib


_f = ctypes.POINTER(ctypes.c_float)
_d = ctypes.POINTER(ctypes.c_double)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_i64 = ctypes.POINTER(ctypes.c_int64)
_u32 = ctypes.POINTER(ctypes.c_uint32)
_i32 = ctypes.POINTER(ctypes.c_int32)


def _declare(L):
    if hasattr(L, "oracle_loglik"):
        _declare_loglik(L)
    if hasattr(L, "oracle_philox4x32_10"):
        _declare_mcmc(L)


def _declare_loglik(L):
    sig = [ctypes.c_int, _f, _f, _f, _f, _f, ctypes.c_int64, _f, _u8, ctypes.c_int]
    for name in ("oracle_loglik", "oracle_loglik_backward", "oracle_loglik_ld",
                 "oracle_loglik_bruteforce"):
        fn = getattr(L, name)
        fn.argtypes = sig
        fn.restype = ctypes.c_double
    L.oracle_log_emission.argtypes = [ctypes.c_int, _f, _f, _f, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_double, _d]
    L.oracle_log_emission.restype = None
    L.oracle_loglik_batched.argtypes = [ctypes.c_int, ctypes.c_int, _f, _f, _f, _f, _f,
                                        ctypes.c_int, _i64, _f, _u8, ctypes.c_int, _d,
                                        ctypes.c_int]
    L.oracle_loglik_batched.restype = None
    L.oracle_posterior.argtypes = [ctypes.c_int, _f, _f, _f, _f, _f, ctypes.c_int64, _f, _u8, ctypes.c_int, _d]
    L.oracle_posterior.restype = ctypes.c_double
    L.oracle_expected_stats.argtypes = [ctypes.c_int, _f, _f, _f, _f, _f, ctypes.c_int64, _f, _u8, ctypes.c_int,
                                        _d]
    L.oracle_expected_stats.restype = ctypes.c_double
    L.oracle_viterbi.argtypes = [ctypes.c_int, _f, _f, _f, _f, _f, ctypes.c_int64, _f, _u8, ctypes.c_int, _i32]
    L.oracle_viterbi.restype = ctypes.c_double
    L.oracle_path_logjoint.argtypes = [ctypes.c_int, _f, _f, _f, _f, _f, ctypes.c_int64, _f, _u8, ctypes.c_int,
                                       _i32]
    L.oracle_path_logjoint.restype = ctypes.c_double


class OraclePrior(ctypes.Structure):
    """Mirror of the oracle's prior settings (see mcmc_oracle.c)."""
    _fields_ = [("alpha_P", ctypes.c_double), ("alpha_pi", ctypes.c_double),
                ("p_mean_lo", ctypes.c_double), ("p_mean_hi", ctypes.c_double),
                ("p_var", ctypes.c_double), ("box", ctypes.c_double * 4),
                ("iw_df", ctypes.c_double)]


def _declare_mcmc(L):
    L.oracle_philox4x32_10.argtypes = [_u32, _u32, _u32]
    L.oracle_philox4x32_10.restype = None
    L.oracle_normal.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                ctypes.c_uint32]
    L.oracle_normal.restype = ctypes.c_double
    L.oracle_uniform.argtypes = L.oracle_normal.argtypes
    L.oracle_uniform.restype = ctypes.c_double
    L.oracle_theta_dim.argtypes = [ctypes.c_int]
    L.oracle_theta_dim.restype = ctypes.c_int
    L.oracle_theta_to_params.argtypes = [ctypes.c_int, _d, ctypes.POINTER(OraclePrior), _d, _d, _d, _d, _d]
    L.oracle_theta_to_params.restype = ctypes.c_double
    if hasattr(L, "oracle_mlp_forward"):
        L.oracle_mlp_forward.argtypes = [ctypes.c_int, ctypes.c_int, _d, _d, _d, ctypes.c_int, _d, _d]
        L.oracle_mlp_forward.restype = None
        L.oracle_mlp_loss_grad.argtypes = [ctypes.c_int, ctypes.c_int, _d, _d, _d, _d, ctypes.c_int, _d, _d, _d]
        L.oracle_mlp_loss_grad.restype = ctypes.c_double
        L.oracle_adam_step.argtypes = [ctypes.c_size_t, _d, _d, _d, _d, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.oracle_adam_step.restype = None
    if hasattr(L, "oracle_twalk_propose"):
        _ip = ctypes.POINTER(ctypes.c_int)
        L.oracle_twalk_propose.argtypes = [ctypes.c_int, _f, _f, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           _ip, _ip, _ip, _f, _d, _d]
        L.oracle_twalk_propose.restype = None
        L.oracle_twalk_gauss_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_uint64, _d, _f, _f, _f, _d]
        L.oracle_twalk_gauss_run.restype = None


def default_prior(K, box=(0.0, 300.0, 0.0, 150.0)):
    """The prior settings read from Section "Model priors" and Appendix A."""
    return dict(alpha_P=0.01, alpha_pi=1.0, p_mean_lo=0.1, p_mean_hi=0.9, p_var=0.001,
                box=tuple(box), iw_df=float(K))


def _prior_struct(prior):
    pr = OraclePrior()
    for k, v in prior.items():
        if k == "box":
            pr.box = (ctypes.c_double * 4)(*v)
        else:
            setattr(pr, k, float(v))
    return pr


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(c.ctypes.data_as(_u32), k.ctypes.data_as(_u32), out.ctypes.data_as(_u32))
    return out


def normal(seed, stream, chain, it, index):
    return lib().oracle_normal(int(seed), int(stream), int(chain), int(it), int(index))


def uniform(seed, stream, chain, it, index):
    return lib().oracle_uniform(int(seed), int(stream), int(chain), int(it), int(index))


def theta_dim(K):
    return int(lib().oracle_theta_dim(int(K)))


def theta_to_params(theta, K, prior):
    """theta -> (pi, P, p, mu, cov) in float64 and log prior + log Jacobian."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    assert th.shape == (theta_dim(K),)
    pi = np.zeros(K); P = np.zeros(K * K); p = np.zeros(K); mu = np.zeros(2 * K); cov = np.zeros(3 * K)
    pr = _prior_struct(prior)
    lp = lib().oracle_theta_to_params(int(K), th.ctypes.data_as(_d), ctypes.byref(pr), pi.ctypes.data_as(_d),
                                      P.ctypes.data_as(_d), p.ctypes.data_as(_d), mu.ctypes.data_as(_d),
                                      cov.ctypes.data_as(_d))
    return (pi, P.reshape(K, K), p, mu.reshape(K, 2), cov.reshape(K, 3)), lp


def compile_variant(source_text: str, out_dir) -> ctypes.CDLL:
    """Compile a modified copy of the oracle source (mutation tests only)."""
    out_dir = Path(out_dir)
    src = out_dir / "variant.c"
    src.write_text(source_text)
    so = out_dir / "libvariant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                    "-o", str(so), str(src), "-lm", "-lpthread"], check=True)
    L = ctypes.CDLL(str(so))
    _declare(L)
    return L


def _fp(a):
    return a.ctypes.data_as(_f)


def _c32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _args(prm, xy, tremor):
    pi, P, p, mu, cov = (_c32(x) for x in prm)
    xy = _c32(xy).reshape(-1, 2)
    tremor = np.ascontiguousarray(np.asarray(tremor, dtype=np.uint8))
    keep = (pi, P, p, mu, cov, xy, tremor)
    return keep, (int(pi.shape[-1]), _fp(pi), _fp(P), _fp(p), _fp(mu), _fp(cov),
                  int(tremor.shape[0]), _fp(xy), tremor.ctypes.data_as(_u8))


def _params(prm):
    return prm.as_tuple() if hasattr(prm, "as_tuple") else tuple(prm)


def loglik(prm, xy, tremor, init_mode: int = 0, _L=None) -> float:
    """Scaled FP64 forward algorithm (Algorithm 1 with scale coefficients)."""
    keep, a = _args(_params(prm), xy, tremor)
    return (_L or lib()).oracle_loglik(*a, int(init_mode))


def loglik_backward(prm, xy, tremor, init_mode: int = 0, _L=None) -> float:
    keep, a = _args(_params(prm), xy, tremor)
    return (_L or lib()).oracle_loglik_backward(*a, int(init_mode))


def loglik_longdouble(prm, xy, tremor, init_mode: int = 0, _L=None) -> float:
    keep, a = _args(_params(prm), xy, tremor)
    return (_L or lib()).oracle_loglik_ld(*a, int(init_mode))


def loglik_bruteforce(prm, xy, tremor, init_mode: int = 0, _L=None) -> float:
    keep, a = _args(_params(prm), xy, tremor)
    return (_L or lib()).oracle_loglik_bruteforce(*a, int(init_mode))


def log_emission(prm, x: float, y: float, tremor: int, _L=None) -> np.ndarray:
    pi, P, p, mu, cov = (_c32(x_) for x_ in _params(prm))
    K = int(p.shape[0])
    out = np.zeros(K, dtype=np.float64)
    (_L or lib()).oracle_log_emission(K, _fp(p), _fp(mu), _fp(cov), int(tremor), float(x), float(y),
                              out.ctypes.data_as(_d))
    return out


def loglik_batched(prm, xy, tremor, offsets, init_mode: int = 0, n_threads: int = 1) -> np.ndarray:
    """Per-proposal sum over segments of log L; ``prm`` arrays are stacked [n_prop, ...]."""
    pi, P, p, mu, cov = (_c32(x) for x in _params(prm))
    n_prop, K = int(pi.shape[0]), int(pi.shape[1])
    xy = _c32(xy).reshape(-1, 2)
    tremor = np.ascontiguousarray(np.asarray(tremor, dtype=np.uint8))
    offs = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    out = np.zeros(n_prop, dtype=np.float64)
    lib().oracle_loglik_batched(n_prop, K, _fp(pi), _fp(P), _fp(p), _fp(mu), _fp(cov),
                                int(offs.shape[0] - 1), offs.ctypes.data_as(_i64), _fp(xy),
                                tremor.ctypes.data_as(_u8), int(init_mode),
                                out.ctypes.data_as(_d), int(n_threads))
    return out


def _dp(a):
    return a.ctypes.data_as(_d)


def _c64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def mlp_num_params(d, H):
    return H * d + H + H * H + H + 2 * d * H + 2 * d


def mlp_forward(params, d, H, mean, in_scale, theta):
    p, m, s, th = _c64(params), _c64(mean), _c64(in_scale), _c64(theta).reshape(-1, d)
    out = np.zeros((th.shape[0], 2 * d))
    lib().oracle_mlp_forward(d, H, _dp(p), _dp(m), _dp(s), th.shape[0], _dp(th), _dp(out))
    return out


def mlp_loss_grad(params, d, H, mean, in_scale, scale, theta, y):
    p, m, si, s = _c64(params), _c64(mean), _c64(in_scale), _c64(scale)
    th, yy = _c64(theta).reshape(-1, d), _c64(y).reshape(-1, d)
    g = np.zeros(mlp_num_params(d, H))
    loss = lib().oracle_mlp_loss_grad(d, H, _dp(p), _dp(m), _dp(si), _dp(s), th.shape[0], _dp(th), _dp(yy),
                                      _dp(g))
    return loss, g


def adam_step(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam step on float64 arrays (returns them)."""
    for a in (params, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oracle_adam_step(params.size, _dp(params), _dp(grad), _dp(m), _dp(v), int(t), lr, b1, b2, eps)
    return params, m, v


TWALK_KERNELS = ("traverse", "walk", "blow", "hop")


def twalk_propose(x, xp, seed, chain, it):
    """One t-walk proposal (twalk_oracle.c): (side, kernel name, n_phi, y float32, W)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    xp = np.ascontiguousarray(np.asarray(xp, dtype=np.float32))
    n = x.size
    y = np.zeros(n, dtype=np.float32)
    work = np.zeros(6 * n + 1, dtype=np.float64)
    side, kern, m = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    W = ctypes.c_double(0.0)
    lib().oracle_twalk_propose(int(n), x.ctypes.data_as(_f), xp.ctypes.data_as(_f), ctypes.c_uint64(seed),
                               ctypes.c_uint32(chain), ctypes.c_uint32(it), ctypes.byref(side), ctypes.byref(kern),
                               ctypes.byref(m), y.ctypes.data_as(_f), ctypes.byref(W),
                               work.ctypes.data_as(_d))
    return side.value, TWALK_KERNELS[kern.value], m.value, y, W.value


TWALK_MIXTURE = (0.4918, 0.9836, 0.9918)


def twalk_gauss_run(x0, xp0, n_iter, seed, kernels=TWALK_MIXTURE, _L=None):
    """A t-walk run on the standard normal target (twalk_oracle.c): samples
    [n_iter, n]. `kernels`: cumulative probabilities of traverse, walk, blow
    (the rest is hop); e.g. (0, 0, 1) runs the blow kernel alone."""
    F = np.ascontiguousarray(np.asarray(kernels, dtype=np.float64))
    x0 = np.ascontiguousarray(np.asarray(x0, dtype=np.float32))
    xp0 = np.ascontiguousarray(np.asarray(xp0, dtype=np.float32))
    n = x0.size
    out = np.zeros((n_iter, n), dtype=np.float32)
    work = np.zeros(6 * n + 2 * n + 2, dtype=np.float64)  # 6n doubles + 3n floats
    (_L or lib()).oracle_twalk_gauss_run(int(n), int(n_iter), ctypes.c_uint64(seed), F.ctypes.data_as(_d),
                                         x0.ctypes.data_as(_f),
                                 xp0.ctypes.data_as(_f), out.ctypes.data_as(_f), work.ctypes.data_as(_d))
    return out


def posterior(prm, xy, tremor, init_mode: int = 0, _L=None):
    """Posterior state probabilities gamma [T, K] (float64) and log L."""
    keep, a = _args(_params(prm), xy, tremor)
    K, T = a[0], a[6]
    g = np.zeros((T, K), dtype=np.float64)
    ll = (_L or lib()).oracle_posterior(*a, int(init_mode), g.ctypes.data_as(_d))
    return g, float(ll)


STAT_NAMES = ("N", "G0", "Gs", "Gr", "Sx", "Sy", "Sxx", "Sxy", "Syy")


def split_stats(flat, K):
    """The flat statistics vector (K*K + 8K) as a dict of arrays."""
    flat = np.asarray(flat)
    out = {"N": flat[:K * K].reshape(K, K)}
    for i, name in enumerate(STAT_NAMES[1:]):
        out[name] = flat[K * K + i * K:K * K + (i + 1) * K]
    return out


def expected_stats(prm, xy, tremor, init_mode: int = 0, _L=None):
    """E-step statistics (dict, float64) and log L (hmm_oracle.c)."""
    keep, a = _args(_params(prm), xy, tremor)
    K = a[0]
    st = np.zeros(K * K + 8 * K, dtype=np.float64)
    ll = (_L or lib()).oracle_expected_stats(*a, int(init_mode), st.ctypes.data_as(_d))
    return split_stats(st, K), float(ll)


def viterbi(prm, xy, tremor, init_mode: int = 0, _L=None):
    """Most probable hidden path (int32 [T]) and its log joint probability."""
    keep, a = _args(_params(prm), xy, tremor)
    T = a[6]
    path = np.zeros(max(T, 1), dtype=np.int32)
    v = (_L or lib()).oracle_viterbi(*a, int(init_mode), path.ctypes.data_as(_i32))
    return path[:T], float(v)


def path_logjoint(prm, xy, tremor, path, init_mode: int = 0):
    """log p(path, observations)."""
    keep, a = _args(_params(prm), xy, tremor)
    path = np.ascontiguousarray(np.asarray(path, dtype=np.int32))
    return float(lib().oracle_path_logjoint(*a, int(init_mode), path.ctypes.data_as(_i32)))
