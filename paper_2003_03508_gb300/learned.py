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


def history_pairs(theta_trace: torch.Tensor, lag: int, burn: int = 0, cross: bool = False, seed: int = 0):
    """Training pairs from a trace [n_iter, C, D] (CUDA float32, contiguous).

    cross=False: (theta_t, theta_{t+lag}) of the same chain,
    [(n_iter-burn-lag)*C] pairs. cross=True: (theta_t of chain c, theta_t of
    chain pi(c)) for a fixed random pairing pi of the chains, [(n_iter-burn)*C]
    pairs -- with many chains spread over the posterior these are close to
    pairs of independent draws, so the network learns the posterior's
    location and spread rather than the random walk's step."""
    tr = theta_trace[burn:]
    if cross:
        g = torch.Generator(device="cpu").manual_seed(seed)
        perm = torch.randperm(tr.shape[1], generator=g).to(tr.device)
        X = tr.reshape(-1, tr.shape[-1]).contiguous()
        Y = tr[:, perm].reshape(-1, tr.shape[-1]).contiguous()
        return X, Y
    X = tr[:-lag].reshape(-1, tr.shape[-1]).contiguous()
    Y = tr[lag:].reshape(-1, tr.shape[-1]).contiguous()
    return X, Y


def acceptance(sampler: api.Sampler, n_iter: int) -> float:
    _, _, _, na0 = sampler.state()
    sampler.step(n_iter)
    _, _, _, na1 = sampler.state()
    return float((na1 - na0).double().mean().item()) / n_iter


def esjd(theta_trace: torch.Tensor, scale: torch.Tensor) -> float:
    """Expected squared jump distance of a trace [n, C, D]: the mean over
    iterations and chains of sum_i ((theta_{t+1} - theta_t)_i / scale_i)^2."""
    d = (theta_trace[1:] - theta_trace[:-1]) / scale
    return float((d * d).sum(dim=2).mean().item())


def pcn_pairs(rhos):
    """(lam, gamma) pairs of the autoregressive family: with the network
    giving the mean m and spread tau of an independent posterior draw (the
    cross-chain training target), the proposal theta + lam gamma (m - theta) +
    lam tau z equals m + rho (theta - m) + sqrt(1 - rho^2) tau z when
    lam = sqrt(1 - rho^2) and gamma = sqrt((1 - rho) / (1 + rho)): for a
    Gaussian posterior with that mean and spread it leaves the posterior
    invariant by itself, so drift and step stay consistent in every dimension
    (a drift without the matching step size is rejected almost always in
    hundreds of dimensions)."""
    return [(float(np.sqrt(1.0 - r * r)), float(np.sqrt((1.0 - r) / (1.0 + r)))) for r in rhos]


def fit_learned_proposal(sampler: api.Sampler, theta_trace: torch.Tensor, lag: int = 20, hidden: int = 256,
                         train_steps: int = 2000, batch: int = 512, lr: float = 2e-3, seed: int = 0,
                         target_accept: float = 0.35, pilot_iters: int = 50, lams=(0.8, 0.4, 0.2, 0.1),
                         gamma: float = 0.5, burn: int = 0, select: str = "accept", gammas=None,
                         cross: bool = False, pairs=None):
    """Train an MLP proposal on a random-walk trace and attach it to `sampler`.

    gamma scales the learned drift (the proposal mean is theta + lam s gamma
    f_mu): a full-strength drift learned from finite history makes the
    reverse move unlikely in many coordinates at once, so it is damped. lam
    is chosen by short pilot runs: select="accept" takes the one whose
    acceptance is closest to target_accept, select="esjd" the one with the
    largest expected squared jump distance in units of the history's
    per-coordinate spread. With `gammas` given, the drift factor is searched
    together with lam (every pair is piloted); with `pairs` given, exactly
    those (lam, gamma) pairs are piloted. Returns (mlp, info) where info
    holds the training losses, the chosen lam and gamma, the pilot statistics
    and the wall time spent.
    """
    t0 = time.perf_counter()
    D = theta_trace.shape[-1]
    X, Y = history_pairs(theta_trace, lag, burn, cross=cross, seed=seed)
    mlp = api.MLP(D, hidden=hidden, seed=seed)
    mlp.fit_scaling(X, Y, lam=1.0)
    losses = mlp.train(X, Y, train_steps, batch=batch, lr=lr, seed=seed + 1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    sampler.set_proposal(mlp)
    pilot = {}
    best, best_score = None, None
    spread = X.std(dim=0) + 1e-12
    if pairs is not None:
        grid = list(pairs)
    else:
        grid = [(lam, gamma) for lam in lams] if gammas is None else [(lam, g) for g in gammas for lam in lams]
    for lam, gam in grid:
        mlp.set_lambda(lam, gam)
        sampler.set_proposal(mlp)  # rebuild the captured iteration with the new lam
        if select == "esjd":
            _, _, _, na0 = sampler.state()
            _, th = sampler.step(pilot_iters, trace_theta=True)
            _, _, _, na1 = sampler.state()
            acc = float((na1 - na0).double().mean().item()) / pilot_iters
            score = esjd(th, spread)
            pilot[f"{lam:.4g}/{gam:.4g}"] = {"accept": acc, "esjd": score}
            del th
        else:
            acc = acceptance(sampler, pilot_iters)
            score = -abs(acc - target_accept)
            pilot[f"{lam:g}/{gam:g}"] = acc
        if best is None or score > best_score:
            best, best_score = (lam, gam), score
    mlp.set_lambda(best[0], best[1])
    sampler.set_proposal(mlp)
    torch.cuda.synchronize()
    info = dict(losses=losses.cpu().numpy(), lam=best[0], gamma=best[1], pilot=pilot, train_seconds=t_train,
                total_seconds=time.perf_counter() - t0, n_pairs=int(X.shape[0]))
    return mlp, info
