"""Fitting the learned proposal from the random walk's own history.

Host-side orchestration of the C ABI (every computation runs in the
library's kernels): run the random-walk sampler and keep its trace, form
pairs (theta_t, theta_{t+lag}) of the same chain, set the network's
standardisation from those pairs, train it with Adam, then pick the step
factor lam by short pilot runs aiming at a target acceptance rate. The
exact likelihood keeps deciding acceptance, so the posterior is unchanged;
the random walk remains both the fallback and the baseline.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import api


def history_pairs(theta_trace: torch.Tensor, lag: int, burn: int = 0):
    """theta_trace [n_iter, C, D] -> X, Y [(n_iter-burn-lag)*C, D] (CUDA float32, contiguous)."""
    tr = theta_trace[burn:]
    X = tr[:-lag].reshape(-1, tr.shape[-1]).contiguous()
    Y = tr[lag:].reshape(-1, tr.shape[-1]).contiguous()
    return X, Y


def acceptance(sampler: api.Sampler, n_iter: int) -> float:
    _, _, _, na0 = sampler.state()
    sampler.step(n_iter)
    _, _, _, na1 = sampler.state()
    return float((na1 - na0).double().mean().item()) / n_iter


def fit_learned_proposal(sampler: api.Sampler, theta_trace: torch.Tensor, lag: int = 20, hidden: int = 256,
                         train_steps: int = 2000, batch: int = 512, lr: float = 2e-3, seed: int = 0,
                         target_accept: float = 0.35, pilot_iters: int = 50, lams=(0.8, 0.4, 0.2, 0.1),
                         gamma: float = 0.5, burn: int = 0):
    """Train an MLP proposal on a random-walk trace and attach it to `sampler`.

    gamma scales the learned drift (the proposal mean is theta + lam s gamma
    f_mu): a full-strength drift learned from finite history makes the
    reverse move unlikely in many coordinates at once, so it is damped; lam
    is the largest step whose pilot acceptance is closest to target_accept.
    Returns (mlp, info) where info holds the training losses, the chosen lam,
    the pilot acceptance rates and the wall time spent.
    """
    t0 = time.perf_counter()
    D = theta_trace.shape[-1]
    X, Y = history_pairs(theta_trace, lag, burn)
    mlp = api.MLP(D, hidden=hidden, seed=seed)
    mlp.fit_scaling(X, Y, lam=1.0)
    losses = mlp.train(X, Y, train_steps, batch=batch, lr=lr, seed=seed + 1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    sampler.set_proposal(mlp)
    pilot = {}
    best = None
    for lam in lams:
        mlp.set_lambda(lam, gamma)
        sampler.set_proposal(mlp)  # rebuild the captured iteration with the new lam
        acc = acceptance(sampler, pilot_iters)
        pilot[lam] = acc
        if best is None or abs(acc - target_accept) < abs(pilot[best] - target_accept):
            best = lam
    mlp.set_lambda(best, gamma)
    sampler.set_proposal(mlp)
    torch.cuda.synchronize()
    info = dict(losses=losses.cpu().numpy(), lam=best, gamma=gamma, pilot=pilot, train_seconds=t_train,
                total_seconds=time.perf_counter() - t0, n_pairs=int(X.shape[0]))
    return mlp, info
