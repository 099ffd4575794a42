"""Host-side helpers for running the samplers: starting states, step sizes,
and the random-walk versus learned-proposal comparison.

Everything that touches the data runs in the library's kernels through
``api``; this module only arranges the calls and summarises the traces.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import api, ess, learned, synth


def theta_from_params(K, pi, P, p_tremor, mu, cov):
    """Inverse of the sampler's parameter transform (host, float64): the
    transformed vector theta of one parameter set. P rows become log-ratios
    to their diagonal entry, pi log-ratios to state 0, p_k logits, mu as is,
    sigma_x, sigma_y logs and rho = cov_xy / (sigma_x sigma_y) its atanh."""
    th = []
    for i in range(K):
        th += [math.log(P[i, j] / P[i, i]) for j in range(K) if j != i]
    th += [math.log(pi[k] / pi[0]) for k in range(1, K)]
    th += [math.log(x / (1.0 - x)) for x in p_tremor]
    th += list(np.asarray(mu, dtype=np.float64).reshape(-1))
    sx, sy = np.sqrt(cov[:, 0]), np.sqrt(cov[:, 2])
    for k in range(K):
        th += [math.log(sx[k]), math.log(sy[k])]
    th += [math.atanh(cov[k, 1] / (sx[k] * sy[k])) for k in range(K)]
    return np.array(th, dtype=np.float64)


def base_steps(K, logit_step=0.05, mean_step_km=2.0):
    """Random-walk step sizes per coordinate: logits and log scales move by
    logit_step, the state means (km) by mean_step_km."""
    D = api.theta_dim(K)
    step = np.full(D, logit_step, np.float32)
    o = K * (K - 1) + (K - 1) + K
    step[o:o + 2 * K] = mean_step_km
    return step


def tremor_problem(K, T, chains, seed, spread=0.01):
    """A synthetic tremor sequence and `chains` starting states near its
    generating parameters (device tensors)."""
    rng = np.random.default_rng(seed)
    gen = synth.random_params(K, rng)
    obs = synth.sample_observations(gen, T, rng)
    base = theta_from_params(K, gen.pi.astype(np.float64), gen.P.astype(np.float64),
                             gen.p_tremor.astype(np.float64), gen.mu.astype(np.float64),
                             gen.cov.astype(np.float64))
    th0 = (base[None, :] + spread * rng.standard_normal((chains, base.size))).astype(np.float32)
    return dict(gen=gen, obs=obs, theta0=torch.from_numpy(th0).cuda(),
                xy=torch.from_numpy(obs.xy).cuda(), tremor=torch.from_numpy(obs.tremor).cuda())


def _timed_run(sampler, n_iter, trace_theta=False):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    lp, th = sampler.step(n_iter, trace_logpost=True, trace_theta=trace_theta)
    e1.record(st)
    torch.cuda.synchronize()
    return lp, th, e0.elapsed_time(e1) / 1e3


def invariant_summaries(theta_trace, K):
    """Label-invariant scalar traces [n_iter, C, 2K] of a theta trace: the
    sorted tremor-probability logits (sorting logits sorts p_k) and the
    sorted x coordinates of the state means."""
    o = K * (K - 1) + (K - 1)
    w = theta_trace[:, :, o:o + K]
    mx = theta_trace[:, :, o + K:o + 3 * K:2]
    return torch.cat([torch.sort(w, dim=2).values, torch.sort(mx, dim=2).values], dim=2)


def _ess_summary(lp, summ, K):
    out = {"log_post": ess.ess_chains(lp.cpu().numpy())}
    summ = summ.cpu().numpy()
    vals = np.array([ess.ess_chains(summ[:, :, j]) for j in range(summ.shape[2])])
    out["summaries_min"] = float(vals.min())
    out["summaries_median"] = float(np.median(vals))
    return out


def rw_vs_learned(K=16, T=16384, chains=512, seed=0, burn=3000, history=200, lag=20, hidden=256,
                  train_steps=2000, batch=512, lr=2e-3, n_measure=1000, alpha_P=0.5,
                  target_accept=0.25, opts=None, cross=True, pilot_iters=100,
                  pcn_rhos=(0.9, 0.97, 0.99, 0.995, 0.998), rw_lams=(0.25, 0.12, 0.06),
                  tune_burn=200, tune_iters=100):
    """Tune and burn in the random walk, train the learned proposal on its
    history (cross=True: pairs of different chains at the same iteration,
    else pairs `lag` iterations apart in one chain), pick its step factor and
    drift factor by the expected squared jump distance of short pilots (the
    autoregressive pairs of learned.pcn_pairs and drift-free steps), then
    run both samplers for n_measure iterations from the same states and
    report effective samples per second of the log posterior and of the
    label-invariant summaries (Geyer initial monotone sequence estimator,
    summed over chains)."""
    # the posterior narrows like 1/sqrt(T): start the chains and the step
    # search at that scale (the defaults were set at T = 16384)
    shrink = min(1.0, math.sqrt(16384.0 / T))
    prob = tremor_problem(K, T, chains, seed, spread=0.01 * shrink)
    pr = api.make_prior(K, alpha_P=alpha_P)
    step0 = base_steps(K) * shrink

    def make(th, step, s):
        return api.Sampler(K, th.contiguous(), torch.from_numpy(step).cuda(), s, [0, T], prob["xy"],
                           prob["tremor"], prior=pr, opts=opts)

    # step multiplier whose acceptance is closest to the target: shrink by
    # sqrt(2) from 1 until the acceptance passes the target (it grows as the
    # step shrinks)
    best = None
    mult = 1.0
    while mult >= 1.0 / 256:
        s = make(prob["theta0"], step0 * mult, seed + 1)
        s.step(tune_burn)
        acc = learned.acceptance(s, tune_iters)
        s.close()
        if best is None or abs(acc - target_accept) < abs(best[1] - target_accept):
            best = (mult, acc)
        if acc >= target_accept:
            break
        mult *= 0.5 ** 0.5
    step = step0 * best[0]
    rw = make(prob["theta0"], step, seed + 2)
    rw.step(burn)
    _, hist, _ = _timed_run(rw, history, trace_theta=True)
    th_now, _, _, _ = rw.state()
    th_early = hist[0].clone()  # each chain's state `history` iterations ago: the t-walk's second point

    t0 = time.perf_counter()
    ls = make(th_now, step, seed + 3)
    mlp, info = learned.fit_learned_proposal(ls, hist, lag=lag, hidden=hidden, train_steps=train_steps,
                                             batch=batch, lr=lr, seed=seed + 4, target_accept=target_accept,
                                             pairs=learned.pcn_pairs(pcn_rhos) + [(lam, 0.0) for lam in rw_lams],
                                             select="esjd", pilot_iters=pilot_iters, cross=cross)
    fit_s = time.perf_counter() - t0
    del hist

    na0 = rw.state()[3].clone()
    lp_rw, th, t_rw = _timed_run(rw, n_measure, trace_theta=True)
    acc_rw = float((rw.state()[3] - na0).double().mean().item()) / n_measure
    sm_rw = invariant_summaries(th, K)
    del th
    na0 = ls.state()[3].clone()
    lp_ml, th, t_ml = _timed_run(ls, n_measure, trace_theta=True)
    acc_ml = float((ls.state()[3] - na0).double().mean().item()) / n_measure
    sm_ml = invariant_summaries(th, K)
    del th
    s_rw = _ess_summary(lp_rw, sm_rw, K)
    s_ml = _ess_summary(lp_ml, sm_ml, K)
    # the t-walk (the paper's sampler) from the same states
    tw = make(th_now, step, seed + 5)
    tw.set_twalk(th_early)
    na0 = tw.state()[3].clone()
    lp_tw, th, t_tw = _timed_run(tw, n_measure, trace_theta=True)
    acc_tw = float((tw.state()[3] - na0).double().mean().item()) / n_measure
    sm_tw = invariant_summaries(th, K)
    del th
    s_tw = _ess_summary(lp_tw, sm_tw, K)
    tw.close()
    e_rw, e_ml = s_rw["log_post"], s_ml["log_post"]
    finite = bool(torch.isfinite(lp_ml).all().item() and torch.isfinite(lp_rw).all().item())
    out = {
        "K": K, "T": T, "chains": chains, "theta_dim": api.theta_dim(K), "iterations": n_measure,
        "burn_in": burn, "history": history, "step_scale": shrink,
        "rw": {"ess": e_rw, "seconds": t_rw, "ess_per_s": e_rw / t_rw, "accept": acc_rw,
               "step_mult": best[0] * shrink, "ms_per_iter": 1e3 * t_rw / n_measure,
               "ess_summaries_min": s_rw["summaries_min"], "ess_summaries_median": s_rw["summaries_median"]},
        "learned": {"ess": e_ml, "seconds": t_ml, "ess_per_s": e_ml / t_ml, "accept": acc_ml,
                    "lam": info["lam"], "gamma": info["gamma"], "hidden": hidden, "lam_pilots": info["pilot"],
                    "ms_per_iter": 1e3 * t_ml / n_measure,
                    "ess_summaries_min": s_ml["summaries_min"], "ess_summaries_median": s_ml["summaries_median"],
                    "ess_per_s_training_amortised": e_ml / (t_ml + fit_s)},
        "twalk": {"ess": s_tw["log_post"], "seconds": t_tw, "ess_per_s": s_tw["log_post"] / t_tw,
                  "accept": acc_tw, "ms_per_iter": 1e3 * t_tw / n_measure,
                  "ess_summaries_min": s_tw["summaries_min"], "ess_summaries_median": s_tw["summaries_median"]},
        "gain_ess_per_s": (e_ml / t_ml) / (e_rw / t_rw),
        "gain_ess_per_iter": e_ml / e_rw,
        "gain_summaries_min_per_s": (s_ml["summaries_min"] / t_ml) / (s_rw["summaries_min"] / t_rw),
        "gain_summaries_median_per_s": (s_ml["summaries_median"] / t_ml) / (s_rw["summaries_median"] / t_rw),
        "training": {"pairs": info["n_pairs"], "pairs_kind": "cross-chain" if cross else f"lag {lag}",
                     "steps": train_steps, "seconds": fit_s,
                     "loss_first": float(np.mean(info["losses"][:20])),
                     "loss_last": float(np.mean(info["losses"][-100:]))},
        "finite": finite,
    }
    rw.close(); ls.close(); mlp.close()
    return out
