"""Sampler traces as Tracer log files (host-side I/O).

Section "Monte Carlo Markov Chains" checks convergence with Tracer (trace
plots and effective sample sizes). Tracer reads tab-separated text: optional
'#' comment lines, a header whose first column is the iteration ("state"),
then one row per stored sample. This module writes the traces that
Sampler.step returns (log posterior [n_iter, C] and theta [n_iter, C, D])
in that form, one file per chain, with theta's coordinates named after the
layout of hmm_theta_dim: P's reference logits, pi's reference logits,
logit p_k, the means, log sigma and atanh rho.
"""
from __future__ import annotations

from pathlib import Path

import numpy as np


def theta_names(K: int) -> list[str]:
    """Column names of theta for K states (K^2 + 6K - 1 of them), in order."""
    names = [f"zP_{i}_{j}" for i in range(K) for j in range(K) if j != i]
    names += [f"zpi_{k}" for k in range(1, K)]
    names += [f"logit_p_{k}" for k in range(K)]
    for k in range(K):
        names += [f"mu_x_{k}", f"mu_y_{k}"]
    for k in range(K):
        names += [f"log_sx_{k}", f"log_sy_{k}"]
    names += [f"atanh_rho_{k}" for k in range(K)]
    return names


def _host(a):
    if a is None:
        return None
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.asarray(a)


def write_tracer_log(path, logpost, theta=None, K: int | None = None, chain: int = 0, first_state: int = 0,
                     every: int = 1, comment: str | None = None) -> Path:
    """Write one chain's trace as a Tracer log.

    logpost: [n_iter, C] (or [n_iter]) log posterior; theta: optional
    [n_iter, C, D] (or [n_iter, D]) states, named by theta_names(K) (K is
    required with theta). Rows are the iterations first_state + every * t.
    Returns the path written.
    """
    lp = _host(logpost).astype(np.float64)
    if lp.ndim == 2:
        lp = lp[:, chain]
    if lp.ndim != 1:
        raise ValueError("logpost must be [n_iter] or [n_iter, C]")
    cols = ["posterior"]
    data = [lp[:, None]]
    if theta is not None:
        th = _host(theta).astype(np.float64)
        if th.ndim == 3:
            th = th[:, chain, :]
        if th.ndim != 2 or th.shape[0] != lp.shape[0]:
            raise ValueError("theta must be [n_iter, D] or [n_iter, C, D] with logpost's n_iter")
        if K is None:
            raise ValueError("K is needed to name theta's columns")
        names = theta_names(K)
        if th.shape[1] != len(names):
            raise ValueError(f"theta has {th.shape[1]} columns, K={K} needs {len(names)}")
        cols += names
        data.append(th)
    rows = np.concatenate(data, axis=1)
    states = first_state + every * np.arange(rows.shape[0], dtype=np.int64)
    path = Path(path)
    with open(path, "w") as f:
        if comment:
            for line in comment.splitlines():
                f.write(f"# {line}\n")
        f.write("state\t" + "\t".join(cols) + "\n")
        for s, r in zip(states, rows):
            f.write(f"{s}\t" + "\t".join(repr(float(v)) for v in r) + "\n")
    return path


def read_tracer_log(path):
    """(column names, states [n] int64, values [n, m] float64) of a Tracer log."""
    header = None
    states, vals = [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.rstrip("\n").split("\t")
            if header is None:
                if parts[0] != "state":
                    raise ValueError("the first column of a Tracer log is 'state'")
                header = parts[1:]
                continue
            if len(parts) != len(header) + 1:
                raise ValueError(f"row with {len(parts)} fields, header has {len(header) + 1}")
            states.append(int(parts[0]))
            vals.append([float(v) for v in parts[1:]])
    if header is None:
        raise ValueError("no header line")
    return header, np.asarray(states, np.int64), np.asarray(vals, np.float64).reshape(len(states), len(header))
