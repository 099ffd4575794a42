"""Python binding of the C ABI in ``include/hmm_gb300.h`` (argument marshalling only).

Every function here checks shapes and dtypes, takes raw device pointers from
torch tensors and calls the library; all arithmetic runs in the library's
CUDA kernels. There is no CPU fallback: if the library cannot be built or
loaded, or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

HMM_OK = 0
HMM_EINVAL = 1
HMM_ECUDA = 2
HMM_ENOMEM = 3
HMM_ENUMERIC = 4
HMM_ETIMEOUT = 5
HMM_EUNSUPPORTED = 6

HMM_PREC_FP32_SIMT = 0
HMM_PREC_TF32 = 1
HMM_PREC_BF16 = 2
HMM_PREC_TF32_SPLIT = 3

HMM_INIT_EMIT_FIRST = 0
HMM_INIT_TRANSITION_FIRST = 1

HMM_PROPOSAL_RW = 0
HMM_PROPOSAL_MLP = 1
HMM_PROPOSAL_TWALK = 2

PRECISIONS = {"fp32": HMM_PREC_FP32_SIMT, "tf32": HMM_PREC_TF32, "bf16": HMM_PREC_BF16,
              "tf32_split": HMM_PREC_TF32_SPLIT}

_ERR_NAMES = {1: "EINVAL", 2: "ECUDA", 3: "ENOMEM", 4: "ENUMERIC", 5: "ETIMEOUT", 6: "EUNSUPPORTED"}


class HMMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"HMM_{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class hmm_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("init_mode", ctypes.c_int32),
                ("chunk_len", ctypes.c_int32), ("renorm_every", ctypes.c_int32),
                ("recheck_fp32", ctypes.c_int32), ("runlen_min", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class hmm_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("pi", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("p_tremor", ctypes.c_void_p), ("mu", ctypes.c_void_p), ("cov", ctypes.c_void_p)]


class hmm_prior(ctypes.Structure):
    _fields_ = [("alpha_P", ctypes.c_float), ("alpha_pi", ctypes.c_float), ("p_mean_lo", ctypes.c_float),
                ("p_mean_hi", ctypes.c_float), ("p_var", ctypes.c_float), ("box", ctypes.c_float * 4),
                ("iw_df", ctypes.c_float)]


class hmm_obs(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int64), ("xy", ctypes.c_void_p), ("tremor", ctypes.c_void_p)]


_lib = None
_lib_lock = threading.Lock()

_VP = ctypes.c_void_p
_I32 = ctypes.c_int32

# name -> (restype, argtypes); exactly the functions declared in include/hmm_gb300.h
SIGNATURES = {
    "hmm_opts_default": (None, [ctypes.POINTER(hmm_opts)]),
    "hmm_measure_fp32_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "hmm_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int]),
    "hmm_destroy": (ctypes.c_int, [_VP]),
    "hmm_last_error": (ctypes.c_char_p, [_VP]),
    "hmm_status": (ctypes.c_int, [_VP, _VP]),
    "hmm_loglik": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                  ctypes.POINTER(hmm_opts), _VP, _VP]),
    "hmm_posterior": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                     ctypes.POINTER(hmm_opts), _VP, _VP, _VP]),
    "hmm_expected_stats": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                          ctypes.POINTER(hmm_opts), _VP, _VP, _VP]),
    "hmm_loglik_grad": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                       ctypes.POINTER(hmm_opts), _VP, _VP, _VP]),
    "hmm_em_step": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                   ctypes.POINTER(hmm_opts), _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "hmm_viterbi": (ctypes.c_int, [_VP, ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs),
                                   ctypes.POINTER(hmm_opts), _VP, _VP, _VP, _VP]),
    "hmm_loglik_batched": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _I32, _VP,
                                          _VP, _VP, ctypes.POINTER(hmm_opts), _VP, _VP]),
    "hmm_loglik_batched_host": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _I32,
                                               _VP, _VP, _VP, ctypes.POINTER(hmm_opts), _VP, _VP]),
    "hmm_last_launch_count": (ctypes.c_int, [_VP]),
    "hmm_last_chunk_len": (ctypes.c_int, [_VP]),
    "hmm_set_call_graphs": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hmm_last_call_graph": (ctypes.c_int, [_VP]),
    "hmm_default_chunk_len": (ctypes.c_int32, [_I32, _I32, _I32, ctypes.c_int64, _I32]),
    "hmm_tune_candidates": (ctypes.c_int, [_I32, _I32, _I32, ctypes.c_int64, _I32, _VP, _I32,
                                           ctypes.POINTER(_I32)]),
    "hmm_autotune_batched": (ctypes.c_int, [_VP, _I32, _I32, _VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP,
                                            ctypes.POINTER(hmm_opts), _I32, _VP, ctypes.POINTER(_I32),
                                            ctypes.POINTER(ctypes.c_double), _VP]),
    "hmm_tune_lookup": (ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, ctypes.c_int64, _I32, ctypes.POINTER(_I32)]),
    "hmm_tune_clear": (ctypes.c_int, []),
    "hmm_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "hmm_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
    "hmm_prior_default": (None, [ctypes.POINTER(hmm_prior), _I32]),
    "hmm_theta_dim": (ctypes.c_int32, [_I32]),
    "hmm_theta_to_params": (ctypes.c_int, [_I32, _I32, _VP, ctypes.POINTER(hmm_prior), _VP, _VP, _VP, _VP, _VP,
                                           _VP, _VP]),
    "hmm_sampler_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _I32, _I32, ctypes.POINTER(hmm_prior),
                                          _VP, _VP, ctypes.c_uint64, _I32, _VP, _VP, _VP,
                                          ctypes.POINTER(hmm_opts), _VP]),
    "hmm_sampler_destroy": (ctypes.c_int, [_VP]),
    "hmm_mcmc_step": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP]),
    "hmm_sampler_recheck": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "hmm_sampler_fp32_report": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "hmm_sampler_save": (ctypes.c_int, [_VP, ctypes.c_char_p, _VP]),
    "hmm_sampler_load": (ctypes.c_int, [_VP, ctypes.c_char_p, _VP]),
    "hmm_sampler_state": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "hmm_sampler_launches_per_iter": (ctypes.c_int, [_VP]),
    "hmm_sampler_graph_active": (ctypes.c_int, [_VP]),
    "hmm_mlp_create": (ctypes.c_int, [ctypes.POINTER(_VP), _I32, _I32, ctypes.c_uint64, _VP]),
    "hmm_mlp_destroy": (ctypes.c_int, [_VP]),
    "hmm_mlp_num_params": (ctypes.c_int64, [_VP]),
    "hmm_mlp_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "hmm_mlp_set_scaling": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_float, _VP]),
    "hmm_mlp_forward": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP]),
    "hmm_mlp_loss_grad": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP]),
    "hmm_mlp_adam_step": (ctypes.c_int, [_VP, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _VP]),
    "hmm_mlp_fit_scaling": (ctypes.c_int, [_VP, _I32, _VP, _VP, ctypes.c_float, _VP]),
    "hmm_mlp_set_lambda": (ctypes.c_int, [_VP, ctypes.c_float, ctypes.c_float]),
    "hmm_mlp_train": (ctypes.c_int, [_VP, _I32, _VP, _VP, _I32, _I32, ctypes.c_float, ctypes.c_uint64, _VP, _VP]),
    "hmm_sampler_set_proposal": (ctypes.c_int, [_VP, _I32, _VP]),
    "hmm_sampler_set_twalk": (ctypes.c_int, [_VP, _VP, _VP]),
    "hmm_sampler_twalk_state": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "hmm_loglik_noalloc": (ctypes.c_int, [ctypes.POINTER(hmm_params), ctypes.POINTER(hmm_obs), _VP, _VP]),
    "hmm_check_bounded_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "hmm_profile_enable": (ctypes.c_int, [_VP, ctypes.c_int]),
    "hmm_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]),
}

PHASES = ("prep", "pack", "chunk", "tree", "final")


def load_library(path=None) -> ctypes.CDLL:
    """Build (if needed) and load the CUDA library; raises if that is impossible."""
    global _lib
    with _lib_lock:
        if _lib is None or path is not None:
            so = path or _build.build()
            L = ctypes.CDLL(str(so))
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            if path is not None:
                return L
            _lib = L
    return _lib


def make_opts(precision="fp32", init_mode=HMM_INIT_EMIT_FIRST, chunk_len=0, renorm_every=0,
              recheck_fp32=0, runlen_min=0) -> hmm_opts:
    """Options for every entry point; runlen_min > 0 turns on the run-length
    shortcut (FP32 only): runs of at least that many no-tremor steps are
    applied as products of precomputed binary powers of P diag(1 - p)."""
    o = hmm_opts()
    load_library().hmm_opts_default(ctypes.byref(o))
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.init_mode = int(init_mode)
    o.chunk_len = int(chunk_len)
    o.renorm_every = int(renorm_every)
    o.recheck_fp32 = int(recheck_fp32)
    o.runlen_min = int(runlen_min)
    return o


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _dev(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


class Context:
    """Owns one ``hmm_ctx`` (workspace, plan cache, device status word)."""

    def __init__(self, device: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the HMM library has no CPU path")
        self.lib = load_library()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = _VP()
        rc = self.lib.hmm_create(ctypes.byref(h), self.device)
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int):
        if rc != HMM_OK:
            raise HMMError(rc, self.lib.hmm_last_error(self.h).decode())

    @property
    def last_launch_count(self) -> int:
        return int(self.lib.hmm_last_launch_count(self.h))

    @property
    def last_chunk_len(self) -> int:
        return int(self.lib.hmm_last_chunk_len(self.h))

    def set_call_graphs(self, on: bool = True):
        """Capture and replay the batched call as a CUDA graph (default on)."""
        self._check(self.lib.hmm_set_call_graphs(self.h, int(bool(on))))

    @property
    def last_call_graph(self) -> int:
        """0: the last call launched its kernels directly; 1: it captured a
        new graph and launched it; 2: it replayed the existing graph."""
        return int(self.lib.hmm_last_call_graph(self.h))

    def hmm_profile_enable(self, on: bool = True):
        self._check(self.lib.hmm_profile_enable(self.h, int(bool(on))))

    def hmm_profile_read(self):
        """(dict phase -> accumulated ms, number of recorded calls)."""
        ms = (ctypes.c_double * len(PHASES))()
        n = ctypes.c_int()
        self._check(self.lib.hmm_profile_read(self.h, ms, ctypes.byref(n)))
        return dict(zip(PHASES, list(ms))), int(n.value)

    def hmm_status(self, stream=None) -> int:
        """Synchronise, read and clear the device status word (returns the code)."""
        return int(self.lib.hmm_status(self.h, _stream_ptr(stream)))

    def hmm_posterior(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, stream=None):
        """Posterior state probabilities [T, K] (float32) and log L (float64 [1]) of one sequence."""
        K = int(pi.shape[0])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        T = int(tremor.shape[0])
        gamma = torch.empty(T, K, dtype=torch.float32, device=pi.device)
        ll = torch.empty(1, dtype=torch.float64, device=pi.device)
        prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(), cov.data_ptr())
        ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
        o = opts if opts is not None else make_opts()
        self._check(self.lib.hmm_posterior(self.h, ctypes.byref(prm), ctypes.byref(ob), ctypes.byref(o),
                                           gamma.data_ptr(), ll.data_ptr(), _stream_ptr(stream)))
        return gamma, ll

    def hmm_expected_stats(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, stream=None):
        """E-step statistics of one sequence as a dict of float64 CUDA tensors
        (N [K, K], G0, Gs, Gr, Sx, Sy, Sxx, Sxy, Syy [K]) and log L."""
        K = int(pi.shape[0])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        T = int(tremor.shape[0])
        flat = torch.empty(K * K + 8 * K, dtype=torch.float64, device=pi.device)
        ll = torch.empty(1, dtype=torch.float64, device=pi.device)
        prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(), cov.data_ptr())
        ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
        o = opts if opts is not None else make_opts()
        self._check(self.lib.hmm_expected_stats(self.h, ctypes.byref(prm), ctypes.byref(ob), ctypes.byref(o),
                                                flat.data_ptr(), ll.data_ptr(), _stream_ptr(stream)))
        out = {"N": flat[:K * K].view(K, K)}
        for i, name in enumerate(("G0", "Gs", "Gr", "Sx", "Sy", "Sxx", "Sxy", "Syy")):
            out[name] = flat[K * K + i * K:K * K + (i + 1) * K]
        return out, ll

    def _one(self, pi, P, p_tremor, mu, cov, xy, tremor, opts):
        K = int(pi.shape[0])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        T = int(tremor.shape[0])
        prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(), cov.data_ptr())
        ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
        o = opts if opts is not None else make_opts()
        return K, prm, ob, o

    def hmm_loglik_grad(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, stream=None):
        """d log L / d(pi, P, p_tremor, mu, cov) as float64 CUDA tensors of the
        parameters' shapes, and log L (float64 [1])."""
        K, prm, ob, o = self._one(pi, P, p_tremor, mu, cov, xy, tremor, opts)
        g = torch.empty(K * K + 7 * K, dtype=torch.float64, device=pi.device)
        ll = torch.empty(1, dtype=torch.float64, device=pi.device)
        self._check(self.lib.hmm_loglik_grad(self.h, ctypes.byref(prm), ctypes.byref(ob), ctypes.byref(o),
                                             g.data_ptr(), ll.data_ptr(), _stream_ptr(stream)))
        cuts = np.cumsum([0, K, K * K, K, 2 * K, 3 * K])
        shapes = ((K,), (K, K), (K,), (K, 2), (K, 3))
        return tuple(g[cuts[i]:cuts[i + 1]].view(*shapes[i]) for i in range(5)), ll

    def hmm_em_step(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, stream=None):
        """One EM iteration: new (pi, P, p_tremor, mu, cov) float32 CUDA
        tensors and log L of the input parameters (float64 [1])."""
        K, prm, ob, o = self._one(pi, P, p_tremor, mu, cov, xy, tremor, opts)
        out = tuple(torch.empty_like(t) for t in (pi, P, p_tremor, mu, cov))
        ll = torch.empty(1, dtype=torch.float64, device=pi.device)
        self._check(self.lib.hmm_em_step(self.h, ctypes.byref(prm), ctypes.byref(ob), ctypes.byref(o),
                                         *(t.data_ptr() for t in out), ll.data_ptr(), _stream_ptr(stream)))
        return out, ll

    def hmm_viterbi(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, stream=None):
        """Most probable hidden path (int32 [T]), its log joint probability and log L (float64 [1] each)."""
        K = int(pi.shape[0])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        T = int(tremor.shape[0])
        path = torch.empty(T, dtype=torch.int32, device=pi.device)
        score = torch.empty(1, dtype=torch.float64, device=pi.device)
        ll = torch.empty(1, dtype=torch.float64, device=pi.device)
        prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(), cov.data_ptr())
        ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
        o = opts if opts is not None else make_opts()
        self._check(self.lib.hmm_viterbi(self.h, ctypes.byref(prm), ctypes.byref(ob), ctypes.byref(o),
                                         path.data_ptr(), score.data_ptr(), ll.data_ptr(), _stream_ptr(stream)))
        return path, score, ll

    def hmm_loglik(self, pi, P, p_tremor, mu, cov, xy, tremor, opts=None, out=None, stream=None):
        """log L of one parameter set on one sequence; returns a float64 [1] CUDA tensor."""
        K = int(pi.shape[0])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        T = int(tremor.shape[0])
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=pi.device)
        prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(),
                         cov.data_ptr())
        ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
        o = opts if opts is not None else make_opts()
        self._check(self.lib.hmm_loglik(self.h, ctypes.byref(prm), ctypes.byref(ob),
                                        ctypes.byref(o), out.data_ptr(), _stream_ptr(stream)))
        return out

    def hmm_loglik_batched(self, pi, P, p_tremor, mu, cov, seg_offsets, xy, tremor, opts=None,
                           out=None, stream=None):
        """Per-proposal sum over segments of log L (float64 [n_prop] CUDA tensor)."""
        n_prop, K = int(pi.shape[0]), int(pi.shape[1])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        offs = np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))
        if out is None:
            out = torch.empty(n_prop, dtype=torch.float64, device=pi.device)
        o = opts if opts is not None else make_opts()
        T = int(offs[-1])
        self._check(self.lib.hmm_loglik_batched(
            self.h, n_prop, K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(),
            cov.data_ptr(), int(offs.shape[0] - 1), offs.ctypes.data,
            xy.data_ptr() if T else None, tremor.data_ptr() if T else None, ctypes.byref(o),
            out.data_ptr(), _stream_ptr(stream)))
        return out

    def hmm_autotune_batched(self, pi, P, p_tremor, mu, cov, seg_offsets, xy, tremor, opts=None,
                             reps=3, out=None, stream=None):
        """Measure the candidate chunk lengths for this shape and store the
        fastest (later calls with chunk_len = 0 use it). Returns
        (out: float64 [n_prop] log L at the winner, chunk length, ms per call)."""
        n_prop, K = int(pi.shape[0]), int(pi.shape[1])
        for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
            _dev(t, torch.float32, n)
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        offs = np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))
        if out is None:
            out = torch.empty(n_prop, dtype=torch.float64, device=pi.device)
        o = opts if opts is not None else make_opts()
        T = int(offs[-1])
        L = ctypes.c_int32(0)
        ms = ctypes.c_double(0.0)
        self._check(self.lib.hmm_autotune_batched(
            self.h, n_prop, K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(),
            cov.data_ptr(), int(offs.shape[0] - 1), offs.ctypes.data,
            xy.data_ptr() if T else None, tremor.data_ptr() if T else None, ctypes.byref(o), int(reps),
            out.data_ptr(), ctypes.byref(L), ctypes.byref(ms), _stream_ptr(stream)))
        return out, int(L.value), float(ms.value)

    def hmm_loglik_batched_host(self, pi, P, p_tremor, mu, cov, seg_offsets, xy, tremor,
                                opts=None, out=None, stream=None):
        """Same as hmm_loglik_batched, with host (numpy or CPU-tensor) inputs and output."""
        def host(a, dt):
            if isinstance(a, torch.Tensor):
                if a.is_cuda:
                    raise TypeError("host entry point takes host buffers")
                if not a.is_contiguous():
                    raise ValueError("host buffers must be contiguous")
                return a, a.data_ptr()
            a = np.ascontiguousarray(a, dtype=dt)
            return a, a.ctypes.data
        keep = []
        ptrs = []
        for a, dt in ((pi, np.float32), (P, np.float32), (p_tremor, np.float32), (mu, np.float32),
                      (cov, np.float32), (xy, np.float32), (tremor, np.uint8)):
            k, ptr = host(a, dt)
            keep.append(k)
            ptrs.append(ptr)
        n_prop, K = int(keep[0].shape[0]), int(keep[0].shape[1])
        offs = np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))
        if out is None:
            out = np.empty(n_prop, dtype=np.float64)
        optr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        o = opts if opts is not None else make_opts()
        self._check(self.lib.hmm_loglik_batched_host(
            self.h, n_prop, K, *ptrs[:5], int(offs.shape[0] - 1), offs.ctypes.data, ptrs[5],
            ptrs[6], ctypes.byref(o), optr, _stream_ptr(stream)))
        return out


def hmm_loglik_noalloc(pi, P, p_tremor, mu, cov, xy, tremor, out=None, stream=None):
    """log L through the allocation-free entry point (no context; fixed scratch).

    Same arguments as Context.hmm_loglik without options; K <= 32, T <= 2^20.
    """
    for t, n in ((pi, "pi"), (P, "P"), (p_tremor, "p_tremor"), (mu, "mu"), (cov, "cov")):
        _dev(t, torch.float32, n)
    _dev(xy, torch.float32, "xy")
    _dev(tremor, torch.uint8, "tremor")
    K = int(pi.shape[0])
    T = int(tremor.shape[0])
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=pi.device)
    prm = hmm_params(K, pi.data_ptr(), P.data_ptr(), p_tremor.data_ptr(), mu.data_ptr(), cov.data_ptr())
    ob = hmm_obs(T, xy.data_ptr() if T else None, tremor.data_ptr() if T else None)
    rc = load_library().hmm_loglik_noalloc(ctypes.byref(prm), ctypes.byref(ob), out.data_ptr(),
                                           _stream_ptr(stream))
    if rc != HMM_OK:
        raise HMMError(rc, "hmm_loglik_noalloc rejected the call")
    return out


def _prec(precision) -> int:
    return PRECISIONS[precision] if isinstance(precision, str) else int(precision)


def chain_steps(seg_offsets) -> int:
    """Total chain steps of a segment layout: sum over segments of max(0, T_s - 1)."""
    T = np.diff(np.asarray(seg_offsets, dtype=np.int64))
    return int(np.maximum(T - 1, 0).sum())


def default_chunk_len(precision, n_prop, K, steps_total, n_sms) -> int:
    """The library's cost-model chunk length for a shape (host only; 0 if out of range)."""
    return int(load_library().hmm_default_chunk_len(_prec(precision), int(n_prop), int(K),
                                                    int(steps_total), int(n_sms)))


def tune_candidates(precision, n_prop, K, steps_total, n_sms) -> list[int]:
    """The chunk lengths the tuner measures for a shape (host only)."""
    buf = (ctypes.c_int32 * 64)()
    n = ctypes.c_int32(0)
    rc = load_library().hmm_tune_candidates(_prec(precision), int(n_prop), int(K), int(steps_total),
                                            int(n_sms), buf, 64, ctypes.byref(n))
    if rc != HMM_OK:
        raise HMMError(rc, "hmm_tune_candidates rejected its arguments")
    return list(buf[:n.value])


def tune_lookup(n_sms, K, precision, n_prop, n_seg, steps_total, runlen_min=0) -> int:
    """Stored chunk length for a shape key, 0 if none (host only)."""
    L = ctypes.c_int32(0)
    rc = load_library().hmm_tune_lookup(int(n_sms), int(K), _prec(precision), int(n_prop), int(n_seg),
                                        int(steps_total), int(runlen_min), ctypes.byref(L))
    if rc != HMM_OK:
        raise HMMError(rc, "hmm_tune_lookup failed")
    return int(L.value)


def tune_clear():
    load_library().hmm_tune_clear()


def tune_save(path):
    rc = load_library().hmm_tune_save(str(path).encode())
    if rc != HMM_OK:
        raise HMMError(rc, f"cannot write the tuning table to {path}")


def tune_load(path):
    rc = load_library().hmm_tune_load(str(path).encode())
    if rc != HMM_OK:
        raise HMMError(rc, f"cannot load a tuning table from {path}")


def make_prior(K, **kw):
    """hmm_prior with the library defaults for K states, fields overridden by kw."""
    pr = hmm_prior()
    load_library().hmm_prior_default(ctypes.byref(pr), int(K))
    for k, v in kw.items():
        if k == "box":
            pr.box = (ctypes.c_float * 4)(*v)
        else:
            setattr(pr, k, float(v))
    return pr


def theta_dim(K):
    return int(load_library().hmm_theta_dim(int(K)))


def theta_to_params(theta, K, prior=None, stream=None):
    """theta [n, D] CUDA float32 -> (pi, P, p_tremor, mu, cov) CUDA tensors and logprior [n] (float64)."""
    _dev(theta, torch.float32, "theta")
    n = int(theta.shape[0])
    dv = theta.device
    pi = torch.empty(n, K, device=dv)
    P = torch.empty(n, K, K, device=dv)
    p = torch.empty(n, K, device=dv)
    mu = torch.empty(n, K, 2, device=dv)
    cov = torch.empty(n, K, 3, device=dv)
    lp = torch.empty(n, dtype=torch.float64, device=dv)
    pr = prior if prior is not None else make_prior(K)
    rc = load_library().hmm_theta_to_params(n, int(K), theta.data_ptr(), ctypes.byref(pr), pi.data_ptr(),
                                            P.data_ptr(), p.data_ptr(), mu.data_ptr(), cov.data_ptr(),
                                            lp.data_ptr(), _stream_ptr(stream))
    if rc != HMM_OK:
        raise HMMError(rc, "hmm_theta_to_params failed")
    return (pi, P, p, mu, cov), lp


class Sampler:
    """n_chains random-walk Metropolis-Hastings chains (wraps hmm_sampler)."""

    def __init__(self, K, theta0, step, seed, seg_offsets, xy, tremor, prior=None, opts=None, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the sampler has no CPU path")
        self.lib = load_library()
        _dev(theta0, torch.float32, "theta0")
        _dev(step, torch.float32, "step")
        _dev(xy, torch.float32, "xy")
        _dev(tremor, torch.uint8, "tremor")
        self.K, self.C, self.D = int(K), int(theta0.shape[0]), int(theta0.shape[1])
        assert self.D == theta_dim(K) and step.shape == (self.D,)
        self._keep = (xy, tremor)  # the sampler reads them for its whole life
        self.offs = np.ascontiguousarray(np.asarray(seg_offsets, dtype=np.int64))
        self.prior = prior if prior is not None else make_prior(K)
        self.opts = opts if opts is not None else make_opts()
        h = _VP()
        T = int(self.offs[-1])
        rc = self.lib.hmm_sampler_create(ctypes.byref(h), torch.cuda.current_device(), self.C, self.K,
                                         ctypes.byref(self.prior), theta0.data_ptr(), step.data_ptr(),
                                         int(seed), int(self.offs.shape[0] - 1), self.offs.ctypes.data,
                                         xy.data_ptr() if T else None, tremor.data_ptr() if T else None,
                                         ctypes.byref(self.opts), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_sampler_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n_iter, trace_logpost=False, trace_theta=False, stream=None):
        """Run n_iter iterations; returns (logpost trace [n, C], theta trace [n, C, D]) or Nones."""
        lp = torch.empty(n_iter, self.C, device="cuda") if trace_logpost else None
        th = torch.empty(n_iter, self.C, self.D, device="cuda") if trace_theta else None
        rc = self.lib.hmm_mcmc_step(self.h, int(n_iter), lp.data_ptr() if lp is not None else None,
                                    th.data_ptr() if th is not None else None, _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_mcmc_step failed")
        return lp, th

    def recheck(self, stream=None):
        """FP32-SIMT log likelihoods of the current states (float64 [C]) and
        the largest difference from the stored values (float64 [1]); the
        stored values are left as they are."""
        ll = torch.empty(self.C, dtype=torch.float64, device="cuda")
        d = torch.empty(1, dtype=torch.float64, device="cuda")
        rc = self.lib.hmm_sampler_recheck(self.h, ll.data_ptr(), d.data_ptr(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_recheck failed")
        return ll, d

    def fp32_report(self, stream=None):
        """The most recent FP32 recheck (values [C], largest difference [1]); NaN before any."""
        ll = torch.empty(self.C, dtype=torch.float64, device="cuda")
        d = torch.empty(1, dtype=torch.float64, device="cuda")
        rc = self.lib.hmm_sampler_fp32_report(self.h, ll.data_ptr(), d.data_ptr(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_fp32_report failed")
        return ll, d

    def save(self, path, stream=None):
        """Write a checkpoint of the sampler's state to `path`."""
        rc = self.lib.hmm_sampler_save(self.h, str(path).encode(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, f"hmm_sampler_save({path}) failed")

    def load(self, path, stream=None):
        """Restore a checkpoint written by save() for the same chains and data."""
        rc = self.lib.hmm_sampler_load(self.h, str(path).encode(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, f"hmm_sampler_load({path}) failed")

    def state(self, stream=None):
        th = torch.empty(self.C, self.D, device="cuda")
        lp = torch.empty(self.C, dtype=torch.float64, device="cuda")
        ll = torch.empty(self.C, dtype=torch.float64, device="cuda")
        na = torch.empty(self.C, dtype=torch.int64, device="cuda")
        rc = self.lib.hmm_sampler_state(self.h, th.data_ptr(), lp.data_ptr(), ll.data_ptr(), na.data_ptr(),
                                        _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_state failed")
        return th, lp, ll, na

    @property
    def launches_per_iter(self):
        return int(self.lib.hmm_sampler_launches_per_iter(self.h))

    @property
    def graph_active(self):
        return bool(self.lib.hmm_sampler_graph_active(self.h))

    def set_proposal(self, mlp=None):
        """Use the learned proposal of `mlp` (an MLP), or the random walk (None)."""
        kind = HMM_PROPOSAL_MLP if mlp is not None else HMM_PROPOSAL_RW
        rc = self.lib.hmm_sampler_set_proposal(self.h, kind, mlp.h if mlp is not None else None)
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_set_proposal failed")
        self._mlp = mlp

    def set_twalk(self, theta2, stream=None):
        """Switch to the t-walk with second points theta2 [C, D] (CUDA float32)."""
        theta2 = theta2.contiguous()
        _dev(theta2, torch.float32, "theta2")
        if tuple(theta2.shape) != (self.C, self.D):
            raise ValueError(f"theta2 must be [{self.C}, {self.D}]")
        rc = self.lib.hmm_sampler_set_twalk(self.h, theta2.data_ptr(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_set_twalk failed")
        self._mlp = None

    def twalk_state(self, stream=None):
        """(second points [C, D], their log posteriors [C]) of a t-walk sampler."""
        th = torch.empty(self.C, self.D, device="cuda")
        lp = torch.empty(self.C, dtype=torch.float64, device="cuda")
        rc = self.lib.hmm_sampler_twalk_state(self.h, th.data_ptr(), lp.data_ptr(), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_sampler_twalk_state failed")
        torch.cuda.synchronize()
        return th, lp


class MLP:
    """The learned proposal's network (wraps hmm_mlp)."""

    def __init__(self, d, hidden=256, seed=0, stream=None):
        self.lib = load_library()
        self.d, self.hidden = int(d), int(hidden)
        h = _VP()
        rc = self.lib.hmm_mlp_create(ctypes.byref(h), self.d, self.hidden, int(seed), _stream_ptr(stream))
        if rc != HMM_OK:
            raise HMMError(rc, "hmm_mlp_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.hmm_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, rc, what):
        if rc != HMM_OK:
            raise HMMError(rc, what)

    @property
    def num_params(self):
        return int(self.lib.hmm_mlp_num_params(self.h))

    def get_params(self, stream=None):
        out = torch.empty(self.num_params, device="cuda")
        self._ok(self.lib.hmm_mlp_params(self.h, out.data_ptr(), 0, _stream_ptr(stream)), "get params")
        return out

    def set_params(self, p, stream=None):
        _dev(p, torch.float32, "params")
        self._ok(self.lib.hmm_mlp_params(self.h, p.data_ptr(), 1, _stream_ptr(stream)), "set params")

    def set_scaling(self, mean, in_scale, scale, lam, stream=None):
        _dev(mean, torch.float32, "mean"); _dev(in_scale, torch.float32, "in_scale")
        _dev(scale, torch.float32, "scale")
        self._ok(self.lib.hmm_mlp_set_scaling(self.h, mean.data_ptr(), in_scale.data_ptr(), scale.data_ptr(),
                                              float(lam), _stream_ptr(stream)), "set scaling")

    def fit_scaling(self, X, Y, lam, stream=None):
        _dev(X, torch.float32, "X"); _dev(Y, torch.float32, "Y")
        self._ok(self.lib.hmm_mlp_fit_scaling(self.h, int(X.shape[0]), X.data_ptr(), Y.data_ptr(), float(lam),
                                              _stream_ptr(stream)), "fit scaling")

    def set_lambda(self, lam, gamma=1.0):
        self._ok(self.lib.hmm_mlp_set_lambda(self.h, float(lam), float(gamma)), "set lambda")

    def forward(self, theta, stream=None):
        _dev(theta, torch.float32, "theta")
        out = torch.empty(theta.shape[0], 2 * self.d, device="cuda")
        self._ok(self.lib.hmm_mlp_forward(self.h, int(theta.shape[0]), theta.data_ptr(), out.data_ptr(),
                                          _stream_ptr(stream)), "forward")
        return out

    def loss_grad(self, theta, y, stream=None):
        _dev(theta, torch.float32, "theta"); _dev(y, torch.float32, "y")
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        g = torch.empty(self.num_params, device="cuda")
        self._ok(self.lib.hmm_mlp_loss_grad(self.h, int(theta.shape[0]), theta.data_ptr(), y.data_ptr(),
                                            loss.data_ptr(), g.data_ptr(), _stream_ptr(stream)), "loss/grad")
        return loss, g

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self._ok(self.lib.hmm_mlp_adam_step(self.h, float(lr), float(beta1), float(beta2), float(eps),
                                            _stream_ptr(stream)), "adam")

    def train(self, X, Y, n_steps, batch=256, lr=1e-3, seed=0, stream=None):
        """n_steps Adam steps on minibatches of (X, Y) pairs; returns the loss trace (CUDA float64)."""
        _dev(X, torch.float32, "X"); _dev(Y, torch.float32, "Y")
        tr = torch.empty(max(1, n_steps), dtype=torch.float64, device="cuda")
        self._ok(self.lib.hmm_mlp_train(self.h, int(X.shape[0]), X.data_ptr(), Y.data_ptr(), int(n_steps),
                                        int(batch), float(lr), int(seed), tr.data_ptr(), _stream_ptr(stream)),
                 "train")
        return tr[:n_steps]


_default_ctx = {}


def default_context() -> Context:
    dev = torch.cuda.current_device()
    if dev not in _default_ctx:
        _default_ctx[dev] = Context(dev)
    return _default_ctx[dev]


def hmm_loglik(*args, **kw):
    return default_context().hmm_loglik(*args, **kw)


def hmm_loglik_batched(*args, **kw):
    return default_context().hmm_loglik_batched(*args, **kw)


def hmm_loglik_batched_host(*args, **kw):
    return default_context().hmm_loglik_batched_host(*args, **kw)


def to_device(prm, device="cuda"):
    """HMMParams (numpy) -> tuple of CUDA float32 tensors (pi, P, p_tremor, mu, cov)."""
    return tuple(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(device)
                 for a in prm.as_tuple())


def measure_fp32_peak(device: int = 0) -> float:
    """Measured FP32 FFMA TFLOP/s of the device (library kernel)."""
    v = ctypes.c_double(0.0)
    rc = load_library().hmm_measure_fp32_peak(int(device), ctypes.byref(v))
    if rc != HMM_OK:
        raise HMMError(rc, "hmm_measure_fp32_peak failed")
    return float(v.value)


def check_bounded_wait(limit_ms: float = 20.0, device: int = 0):
    """Run the device-side bounded-wait check; returns (status code, ms waited)."""
    w = ctypes.c_double(0.0)
    rc = load_library().hmm_check_bounded_wait(int(device), float(limit_ms), ctypes.byref(w))
    return int(rc), float(w.value)
