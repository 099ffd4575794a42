"""Benchmark: batched tremor-HMM log-likelihood evaluations per second.

Workload (one "step"): n_prop = 256 parameter proposals, each a random-walk
perturbation of one generating parameter set, evaluated on one synthetic
tremor-shaped sequence of T = 2^20 observations with K = 32 hidden states --
one call of hmm_loglik_batched, i.e. every stage of the likelihood path
(parameter constants, observation packing, chunk products, product tree,
FP64 combine). Inputs are resident in HBM when the timed region starts; the
L2 is flushed (a 256 MiB write) between timed steps, outside the events.
Before the warm-up the chunk length is tuned for this shape by the library's
autotuner (hmm_autotune_batched, untimed); the timed calls use the stored
length (chunk_len = 0).

Also reported on the same line:
  plain_gpu     the same metric with the FP32-SIMT chunk products (same
                workload, all proposals);
  tf32_split    the same metric with TF32 chunk products whose P is carried
                as hi + lo (two MMAs): FP32-like accuracy on the tensor cores;
  e2e           the same metric through hmm_loglik_batched_host (pinned host
                buffers, host->device inputs and device->host results inside
                the timed region);
  roofline      the chunk-product kernel against its peak;
  cpu_baseline  the FP64 CPU oracle on a bounded sample, on the host cores;
  runlen        the run-length shortcut (FP32, not in the paper) on a
                sparse-tremor workload of the same size (tremor probabilities
                0.002-0.05, long no-tremor runs) beside the tensor-core path on
                the same data; its arithmetic depends on the data, so it is
                reported apart from the roofline;
  mcmc          effective samples per second of the log posterior and of
                label-invariant summaries: the random-walk sampler, the learned
                (MLP) proposal trained on the random walk's own history, and
                the t-walk, same chains and iterations (K=16, 512 chains,
                T=2^20: the learned-proposal workload; 600 measured iterations
                per sampler after a shortened burn-in so the leg stays within
                a few minutes).

``--impl reference`` times the CPU oracle instead (rank 0 only).
Multi-GPU (torchrun): every rank evaluates its own n_prop proposals (weak
scaling, no data-path collective); value = all ranks' evaluations / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "log-lik evals/s (K=32,T=2^20) batched TC vs plain GPU; ESS/s learned vs RW"
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32")
    ap.add_argument("--K", type=int, default=32)
    ap.add_argument("--T", type=int, default=1 << 20)
    ap.add_argument("--n-prop", type=int, default=256)
    ap.add_argument("--chunk-len", type=int, default=0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip measuring the candidate chunk lengths (hmm_autotune_batched) before the timed steps")
    ap.add_argument("--no-split", action="store_true", help="skip the TF32-split (P as hi + lo) sub-line")
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-mcmc", action="store_true")
    ap.add_argument("--no-runlen", action="store_true")
    ap.add_argument("--runlen-min", type=int, default=4)
    ap.add_argument("--no-peaks", action="store_true")
    ap.add_argument("--mcmc-K", type=int, default=16)
    ap.add_argument("--mcmc-T", type=int, default=1 << 20)
    ap.add_argument("--mcmc-chains", type=int, default=512)
    ap.add_argument("--mcmc-iters", type=int, default=600)
    ap.add_argument("--mcmc-burn", type=int, default=400)
    ap.add_argument("--mcmc-precision", default="tf32_split")
    return ap.parse_args()


def max_over_ranks(x_ms, world, device):
    """The job's time is the slowest rank's: all-reduce MAX (identity on one rank)."""
    if world == 1:
        return float(x_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, total_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1e3)


def rank_seed(seed, rank):
    """Each rank evaluates its own proposals (weak scaling, no data exchange)."""
    return seed + 1000 * rank


def measured_peaks(device):
    """This GPU's FP32 FFMA rate (library kernel) and cuBLAS TF32 GEMM rate
    (torch.matmul with TF32 allowed, 8192^3, best of 10 after warm-up)."""
    import torch
    from paper_2003_03508_gb300 import api
    out = {"fp32_ffma_tflops": api.measure_fp32_peak(device)}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda")
        b = torch.randn(n, n, device="cuda")
        for _ in range(3):
            a @ b
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out["tf32_cublas_tflops"] = 2.0 * n ** 3 / (best / 1e3) / 1e12
        del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# nominal dense tensor rates relative to bf16 (2.25 PF): tf32 1.1 PF
NOMINAL_RATIO = {"tf32": 1.1 / 2.25, "tf32_split": 1.1 / 2.25, "bf16": 1.0}


def roofline_peak(precision, pk):
    d, src = pk
    if precision == "fp32":
        # 152 SMs x 128 FP32 lanes x 2 flop (FFMA) x max SM clock
        mhz = float(d.get("sm_max_mhz", 2070.0))
        return "alu", 152 * 128 * 2 * mhz * 1e6 / 1e12, f"derived: 152 SM x 128 FFMA x 2 x {mhz:.0f} MHz"
    ratio = NOMINAL_RATIO[precision]
    sus = float(d.get("bf16_tflops_sustained", d.get("bf16_tflops")))
    return "tensor", sus * ratio, f"{src} bf16 sustained {sus} x nominal {precision}/bf16 ratio {ratio:.4f}"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.out.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(inputs, n_sample, cores):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    prm = inputs["params"]
    sub = type(prm)(*(a[:n_sample] for a in prm.as_tuple()))
    t0 = time.perf_counter()
    ref = oracle.loglik_batched(sub, inputs["xy"], inputs["tremor"], inputs["offsets"], n_threads=cores)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt, np.asarray(ref, dtype=np.float64)


def workload_config(args, n_seg=1):
    """The workload as both arms name it in `config`."""
    return {"workload": f"tremor HMM log-likelihood, K={args.K}, T={args.T}, "
                        f"{args.n_prop} proposals batched per GPU",
            "K": args.K, "T": args.T, "n_prop": args.n_prop, "n_seg": n_seg}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2003_03508_gb300 import synth
    cores = os.cpu_count() or 1
    inputs = synth.batched_inputs(K=args.K, T=args.T, n_prop=cores, seed=args.seed)
    for _ in range(args.warmup):
        cpu_baseline(inputs, cores, cores)
    times = []
    for _ in range(args.steps):
        _, dt, _ = cpu_baseline(inputs, cores, cores)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    value = cores / (ms / 1e3)
    sample = (f"{cores} of the {args.n_prop} proposals per step, full T={args.T} (K={args.K}), "
              f"one proposal per core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def _quiet_runs(tremor, offsets):
    """Lengths of the maximal no-tremor runs among the chain steps (a
    segment's first observation is not a chain step)."""
    out = []
    for s in range(len(offsets) - 1):
        fl = np.asarray(tremor[offsets[s] + 1:offsets[s + 1]], np.int64)
        z = np.concatenate([[1], fl, [1]])
        out.append(np.diff(np.flatnonzero(z)) - 1)
    r = np.concatenate(out) if out else np.zeros(0, np.int64)
    return r[r > 0]


def runlen_leg(args, api, synth, ctx, stream, flush, world, rank):
    import torch
    d = synth.batched_inputs(K=args.K, T=args.T, n_prop=args.n_prop, seed=rank_seed(args.seed + 100, rank),
                             sparse=True)
    dev = api.to_device(d["params"])
    xy = torch.from_numpy(d["xy"]).cuda()
    fl = torch.from_numpy(d["tremor"]).cuda()
    offs = d["offsets"]
    res = {"workload": f"sparse-tremor HMM log-likelihood, K={args.K}, T={args.T}, {args.n_prop} proposals, "
                       f"tremor probabilities U{synth.SPARSE_P_RANGE}",
           "runlen_min": args.runlen_min, "unit": UNIT}

    def timed(opts, reps=3):
        o = torch.empty(args.n_prop, dtype=torch.float64, device="cuda")
        ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=opts, out=o)
        torch.cuda.synchronize()
        ms = 0.0
        for i in range(reps):
            flush.fill_(i & 0xff)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=opts, out=o)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        ms = max_over_ranks(ms, world, "cuda") / reps
        return ms, o

    rms, rout = timed(api.make_opts(precision="fp32", runlen_min=args.runlen_min))
    res["value"] = world * args.n_prop / (rms / 1e3)
    res["ms_per_step"] = rms
    res["launches_per_step"] = ctx.last_launch_count
    tms, tout = timed(api.make_opts(precision=args.precision))
    res["tc_same_data"] = {"precision": args.precision, "value": world * args.n_prop / (tms / 1e3),
                           "ms_per_step": tms}
    res["speedup_vs_tc"] = tms / rms
    # the arithmetic the shortcut saves, counted on the host (runs are not
    # cut at chunk boundaries here, so this slightly overstates the saving)
    runs = _quiet_runs(d["tremor"], offs)
    steps = int(offs[-1]) - (len(offs) - 1)
    long = runs[runs >= args.runlen_min]
    pops = sum(bin(int(n)).count("1") for n in long)
    res["chain_steps"] = steps
    res["steps_in_long_runs"] = int(long.sum())
    res["matrix_products_per_eval_approx"] = int(steps - long.sum() + pops)
    res["mean_quiet_run"] = float(runs.mean()) if runs.size else 0.0
    res["max_abs_diff_vs_tc"] = float((rout - tout).abs().max().item())
    res["max_rel_diff_vs_tc"] = float(((rout - tout).abs() / tout.abs()).max().item())
    return res


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2003_03508_gb300 import api, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    inputs = synth.batched_inputs(K=args.K, T=args.T, n_prop=args.n_prop, seed=rank_seed(args.seed, rank))
    ctx = api.Context(local)
    dev = api.to_device(inputs["params"])
    xy = torch.from_numpy(inputs["xy"]).cuda()
    fl = torch.from_numpy(inputs["tremor"]).cuda()
    offs = inputs["offsets"]
    opts = api.make_opts(precision=args.precision, chunk_len=args.chunk_len)
    out = torch.empty(args.n_prop, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    steps_per_eval = int(offs[-1]) - (len(offs) - 1)
    flops_per_eval = 2.0 * args.K ** 3 * steps_per_eval

    def step():
        ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=opts, out=out)

    tuned = None
    if not args.no_autotune and args.chunk_len == 0:
        # untimed: the tuner stores the fastest chunk length for this shape and
        # the automatic choice (chunk_len = 0) in the timed steps uses it
        _, tL, tms = ctx.hmm_autotune_batched(*dev, offs, xy, fl, opts=opts, reps=3, out=out)
        tuned = {"chunk_len": tL, "ms_per_call": tms,
                 "candidates": api.tune_candidates(args.precision, args.n_prop, args.K, steps_per_eval,
                                                   torch.cuda.get_device_properties(local).multi_processor_count),
                 "model_choice": api.default_chunk_len(args.precision, args.n_prop, args.K, steps_per_eval,
                                                       torch.cuda.get_device_properties(local).multi_processor_count)}

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches_per_step = ctx.last_launch_count
    L = ctx.last_chunk_len

    sampler = ClockSampler(local)
    sampler.start()
    ctx.hmm_profile_enable(True)
    barrier()
    torch.cuda.synchronize()
    evs = []
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    prof, ncalls = ctx.hmm_profile_read()
    ctx.hmm_profile_enable(False)
    total_ms = max_over_ranks(sum(step_ms), world, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_rate(args.n_prop * args.steps, world, total_ms)
    status = ctx.hmm_status()

    # roofline of the chunk-product kernel (its phase is one launch per step)
    chunk_ms = prof["chunk"] / max(1, ncalls)
    bound, peak, peak_src = roofline_peak(args.precision, peaks())
    achieved = flops_per_eval * args.n_prop / (chunk_ms / 1e3) / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "chunk_traffic.json")
    if os.path.exists(tpath):
        from paper_2003_03508_gb300 import build as _b
        with open(tpath) as f:
            tr = json.load(f)
        key = f"{args.precision}:K{args.K}:T{args.T}:P{args.n_prop}:L{L}"
        ent = tr.get(key)
        if ent and ent.get("kernel_digest") == _b.kernel_digest("hmm_chunk_tc.cu", "hmm_chunk_simt.cu", "hmm_tc_common.cuh"):
            traffic = ent["bytes_per_launch"]
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": "hmm chunk products",
            "peak_source": peak_src, "kernel_ms": chunk_ms,
            "phase_share": {k: v / max(1e-9, sum(prof.values())) for k, v in prof.items()}}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {**workload_config(args, len(offs) - 1),
                   "precision": args.precision, "chunk_len": L,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "chunk_len_source": "autotuned" if tuned else ("fixed" if args.chunk_len else "cost model")},
        "roofline": roof,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "status": status,
    }
    if tuned:
        result["autotune"] = tuned

    def timed_variant(precision, reps=2):
        """The same workload and proposals with other chunk products (untimed
        warm-up call, then `reps` event-timed calls, L2 flushed before each)."""
        vo = api.make_opts(precision=precision)
        vout = torch.empty(args.n_prop, dtype=torch.float64, device="cuda")
        ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=vo, out=vout)
        torch.cuda.synchronize()
        ms = 0.0
        for i in range(reps):
            flush.fill_(i & 0xff)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.hmm_loglik_batched(*dev, offs, xy, fl, opts=vo, out=vout)
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        ms = max_over_ranks(ms, world, "cuda") / reps
        return {"value": job_rate(args.n_prop, world, ms), "unit": UNIT, "precision": precision,
                "n_prop": args.n_prop, "ms_per_step": ms, "chunk_len": ctx.last_chunk_len}, vout

    # plain GPU (FP32-SIMT chunk products) on the same workload and proposals
    variant_out = {}
    if not args.no_plain and args.precision != "fp32":
        result["plain_gpu"], pout = timed_variant("fp32")
        result["plain_gpu"]["precision"] = "fp32_simt"
        result["plain_gpu"]["max_abs_diff_vs_tc"] = float((out - pout).abs().max().item())
        variant_out["plain_gpu"] = pout.cpu().numpy()
    # TF32 with P carried as hi + lo (two MMAs): the tensor-core figure at FP32-like accuracy
    if not args.no_split and args.precision == "tf32":
        result["tf32_split"], sout = timed_variant("tf32_split")
        variant_out["tf32_split"] = sout.cpu().numpy()

    # run-length shortcut on the sparse-tremor workload of the same size
    if not args.no_runlen:
        result["runlen"] = runlen_leg(args, api, synth, ctx, stream, flush, world, rank)

    # end to end through the host-buffer entry point
    if not args.no_e2e:
        hp = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in inputs["params"].as_tuple()]
        hxy = torch.from_numpy(inputs["xy"]).pin_memory()
        hfl = torch.from_numpy(inputs["tremor"]).pin_memory()
        hout = torch.empty(args.n_prop, dtype=torch.float64).pin_memory()
        ctx.hmm_loglik_batched_host(*hp, offs, hxy, hfl, opts=opts, out=hout)
        n_e2e = max(3, args.steps // 2)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_e2e):
            ctx.hmm_loglik_batched_host(*hp, offs, hxy, hfl, opts=opts, out=hout)
        e1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1), world, "cuda")
        h2d = sum(a.numel() * a.element_size() for a in hp) + hxy.numel() * 4 + hfl.numel()
        result["e2e"] = {"value": job_rate(args.n_prop * n_e2e, world, ems), "unit": UNIT,
                         "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8 * args.n_prop,
                         "steps": n_e2e, "ms_per_step": ems / n_e2e,
                         "matches_device_result": bool(np.array_equal(hout.numpy(), out.cpu().numpy()))}

    if rank == 0 and not args.no_peaks:
        pm = measured_peaks(local)
        result["peaks_measured"] = pm
        if args.precision in ("tf32", "tf32_split"):
            result["roofline"]["frac_vs_measured_tf32_cublas"] = achieved / pm["tf32_cublas_tflops"]

    if rank == 0 and not args.no_mcmc:
        from paper_2003_03508_gb300 import chains
        mopts = api.make_opts(precision=args.mcmc_precision, recheck_fp32=1)
        result["mcmc"] = chains.rw_vs_learned(K=args.mcmc_K, T=args.mcmc_T, chains=args.mcmc_chains,
                                              seed=args.seed, n_measure=args.mcmc_iters, opts=mopts,
                                              burn=args.mcmc_burn, pilot_iters=30, tune_burn=100, tune_iters=50,
                                              train_steps=1000)
        result["mcmc"]["likelihood"] = (f"{args.mcmc_precision} tensor cores for every Metropolis-Hastings ratio; "
                                        "the chains' current states (their last accepted proposals) re-evaluated "
                                        "in fp32 at the end of each call into a separate report")

    if rank == 0 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        n_sample = min(args.n_prop, cores)
        v, dt, ref = cpu_baseline(inputs, n_sample, cores)
        result["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": min(cores, n_sample), "kind": "oracle",
                                  "sample": f"{n_sample} of the {args.n_prop} proposals, full T={args.T}, "
                                            f"one proposal per thread ({dt:.1f} s wall)"}
        # log-likelihood error of the timed path against the FP64 oracle on that sample
        got = out[:n_sample].cpu().numpy()
        rel = np.abs(got - ref) / np.abs(ref)
        result["error_vs_oracle"] = {"dtype": args.precision, "proposals": int(n_sample),
                                     "max_rel": float(rel.max()), "max_abs": float(np.abs(got - ref).max()),
                                     "log_lik_mean": float(ref.mean())}
        for name, vals in variant_out.items():
            relv = np.abs(vals[:n_sample] - ref) / np.abs(ref)
            result[name]["max_rel_vs_oracle"] = float(relv.max())
            result[name]["max_abs_vs_oracle"] = float(np.abs(vals[:n_sample] - ref).max())
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


if __name__ == "__main__":
    main()
