#!/usr/bin/env python3
"""Benchmark: batched LJ38 Basin Hopping on GB300 (one JSON line on stdout).

Workload: LJ38 (eps = sigma = 1), 64 independent walkers x K = 8 candidates
per BH step (512 local minimisations per BH step), 500 BH steps, starts
uniform in a cube of side 3.2 sigma (seeded), minimised once before timing;
perturbations +-step per coordinate from Philox (initial step 0.4 sigma,
adapted every 10 steps toward 50% acceptance), kT = 0.8, L-BFGS m = 10 to
||grad E||_inf < 1e-6.  One bench "step" is one bh_step_batched launch that
advances every walker by one adaptation window (10 BH steps = 5120 local
minimisations); the default 50 steps run the workload's 500 BH steps.

metric  converged LJ minimisations per second (minimisations that reached
        ||grad E||_inf < 1e-6 with an FP64 gradient), mixed precision path;
        the FP64 path is measured on the same workload for comparison.
Timing  CUDA events around each step's launch on the launching stream, L2
        flushed (256 MiB write) between steps outside the events; e2e adds,
        every step, the host->device copy of the walker state from pinned
        memory and the device->host copy of the updated state.
N > 1   (torchrun) each rank runs its own 64 walkers (global walker indices
        offset by rank): weak scaling, no collective on the data path.
--impl reference   the FP64 CPU oracle on this host's cores, same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ATOMS, WALKERS, K = 38, 64, 8
BH_PER_LAUNCH = 10          # BH steps per bench step (one adaptation window)
SIDE, STEP0, KT = 3.2, 0.4, 0.8
# MIXED precision policy parameter of this workload: the FP32 tier's gradient
# threshold (swept on LJ38 BH: 1e-3 168k, 3e-4 179k, 1e-4 183k converged/s)
SWITCH_GTOL = 1e-4
CONFIG_ID = 1
WORKLOAD = ("LJ38 Basin Hopping: 64 walkers x K=8 candidates per BH step (512 L-BFGS "
            "minimisations per BH step), 10 BH steps per bench step, cube starts side "
            "3.2 sigma, m=10, ||g||_inf<1e-6")
PAIRS = N_ATOMS * (N_ATOMS - 1) // 2
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e-3   # SMs x FP32 lanes x 2 (FMA) x max SM GHz
FP64_PEAK_TFLOPS = 1.25                    # nominal FP64 (non-tensor) rate of GB300
# dram__bytes_read.sum + dram__bytes_write.sum of one bh_cluster_kernel launch of this
# workload (ncu capture summarised in profiles/bh_cluster_kernel_lj38_64x8.md); set to
# None whenever the kernel changes until it is captured again
BH_DRAM_BYTES_PER_LAUNCH = None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-micro", action="store_true", help="skip the evaluation microbench")
    ap.add_argument("--workload", default="lj38-bh",
                    choices=["lj38-bh", "uneven-4096", "large-500", "large-1000", "lj13-seq"],
                    help="lj38-bh (default): the Basin Hopping step this bench reports; the "
                         "others time the batched minimisation of the uneven and large-cluster "
                         "workloads, or one sequential FP64 LJ13 walker, and print their own line")
    ap.add_argument("--micro-only", action="store_true",
                    help="run only the evaluation microbench and print its JSON")
    ap.add_argument("--micro-repeats", type=int, default=100)
    ap.add_argument("--profile", action="store_true",
                    help="mixed-precision steps only (no FP64 arm, e2e or CPU legs): the "
                         "command to run under ncu; numbers printed then are not bench values")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def start_state(rank):
    from paper_2510_25938_gb300 import inputs as I
    seed = I.workload_seed(CONFIG_ID)
    x0 = I.cube_starts(WALKERS * (rank + 1), N_ATOMS, SIDE, seed)[WALKERS * rank:]
    return x0, seed


def flops_from_stats(s):
    """Algorithmic flops: 28 per unordered pair per evaluation, and per
    L-BFGS iteration 8 * (history pairs used) * 3N (two dots + two axpys per
    pair) + 12 * 3N for the remaining vector updates."""
    pair = 28.0 * (s["pairs32"] + s["pairs64"] + s["pairs_df"])
    vec = 8.0 * (s["vec_elems32"] + s["vec_elems64"]) + 12.0 * 3 * N_ATOMS * (
        s["iters32"] + s["iters64"])
    return pair + vec, 28.0 * (s["pairs64"] + s["pairs_df"])


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def cpu_baseline(x0, seed, budget_s=12.0):
    """The FP64 oracle on this host's cores: BH steps of all 64 walkers, as
    many as fit in ~budget_s (at least one)."""
    import oracle as O
    xm, em, st, _, _ = O.lbfgs_batch(x0, x0.shape[0], uniform_n=N_ATOMS)
    xm = xm.reshape(x0.shape[0], -1)
    state = {"x_cur": xm.copy(), "e_cur": em.copy(), "x_best": xm.copy(), "e_best": em.copy(),
             "stepsize": np.full(x0.shape[0], STEP0), "win_accept": np.zeros(x0.shape[0], np.int32),
             "n_accept": np.zeros(x0.shape[0], np.int32)}
    conv = mins = 0
    steps = 0
    t0 = time.perf_counter()
    while steps == 0 or time.perf_counter() - t0 < budget_s:
        tr = O.bh_run(state, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=steps, n_steps=1))
        conv += int((tr["trial_status"] == O.CONVERGED).sum())
        mins += tr["trial_status"].size
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": conv / dt, "unit": "converged minimisations/s", "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"{steps} BH steps x 64 walkers x K=8 = {mins} FP64 minimisations of LJ38 "
                      f"({conv} converged) in {dt:.1f} s"}


def eval_microbench(L, ctx, dev, flush, repeats=100):
    """Energy+gradient throughput on 65,536 LJ38 configurations: 1,024 local
    minima (GPU FP64 minimiser from seeded cube starts of side 3.2 sigma) x 64
    Gaussian jitters (sigma_x = 0.05 sigma), FP32 and FP64, `repeats` timed
    sweeps each with L2 flushed between sweeps; pair evaluations per second
    (703 unordered pairs per configuration) and algorithmic TFLOP/s
    (28 flops per pair) against the FP32 / FP64 non-tensor peaks."""
    import torch
    from paper_2510_25938_gb300 import inputs as I
    seed = I.workload_seed(2)
    x0 = I.cube_starts(1024, N_ATOMS, SIDE, seed)
    x = torch.as_tensor(x0.reshape(-1), dtype=torch.float64, device=dev).contiguous()
    e = torch.empty(1024, dtype=torch.float64, device=dev)
    L.lbfgs_minimize_batched(ctx, x, e, n_cand=1024, uniform_n=N_ATOMS,
                             params=L.LbfgsParams(prec=L.LJ_PREC_FP64))
    minima = x.view(1024, -1).cpu().numpy()
    cfg = I.jitter(np.repeat(minima, 64, axis=0), 0.05, seed + 1)
    n_cand = cfg.shape[0]
    pairs = n_cand * PAIRS
    out = {"configs": n_cand, "repeats": repeats, "pairs_per_sweep": pairs}
    stream = torch.cuda.current_stream()
    for name, dt, prec, peak in (("fp32", torch.float32, L.LJ_PREC_FP32, FP32_PEAK_TFLOPS),
                                 ("fp64", torch.float64, L.LJ_PREC_FP64, FP64_PEAK_TFLOPS)):
        xd = torch.as_tensor(cfg.reshape(-1), dtype=dt, device=dev).contiguous()
        en = torch.empty(n_cand, dtype=torch.float64, device=dev)
        gr = torch.empty_like(xd)
        for _ in range(3):
            L.lj_energy_grad_batched(ctx, xd, en, gr, n_cand=n_cand, uniform_n=N_ATOMS, prec=prec)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(repeats)]
        torch.cuda.synchronize()
        for r in range(repeats):
            flush.fill_(float(r))
            ev[r][0].record(stream)
            L.lj_energy_grad_batched(ctx, xd, en, gr, n_cand=n_cand, uniform_n=N_ATOMS, prec=prec)
            ev[r][1].record(stream)
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        rate = pairs * repeats / t
        out[name] = {"pair_evals_per_s": rate, "ms_per_sweep": 1e3 * t / repeats,
                     "achieved_tflops": 28.0 * rate / 1e12, "peak_tflops": peak,
                     "frac": 28.0 * rate / 1e12 / peak,
                     "hbm_gbs": (xd.numel() * xd.element_size() * 2 + 8 * n_cand) * repeats / t / 1e9}
    out["peaks"] = "FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz; FP64: nominal 1.25 TFLOP/s"
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    x0, seed = start_state(0)
    import oracle as O
    xm, em, st, _, _ = O.lbfgs_batch(x0, WALKERS, uniform_n=N_ATOMS)
    xm = xm.reshape(WALKERS, -1)
    state = {"x_cur": xm.copy(), "e_cur": em.copy(), "x_best": xm.copy(), "e_best": em.copy(),
             "stepsize": np.full(WALKERS, STEP0), "win_accept": np.zeros(WALKERS, np.int32),
             "n_accept": np.zeros(WALKERS, np.int32)}
    # each reference step is a bounded sample: one BH step of all 64 walkers
    # (1/10 of a bench step's work), so that --steps K --warmup W ends in minutes
    for s in range(args.warmup):
        O.bh_run(state, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=s, n_steps=1))
    conv = mins = 0
    t0 = time.perf_counter()
    for s in range(args.steps):
        tr = O.bh_run(state, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=args.warmup + s,
                                          n_steps=1))
        conv += int((tr["trial_status"] == O.CONVERGED).sum())
        mins += tr["trial_status"].size
    dt = time.perf_counter() - t0
    v = conv / dt
    line = {"metric": "converged LJ minimisations/s", "value": v,
            "unit": "converged minimisations/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps * BH_PER_LAUNCH,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "converged minimisations/s",
                             "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} BH steps x 64 walkers x K=8 = {mins} "
                                       f"FP64 minimisations ({conv} converged); "
                                       f"ms_per_step scaled to 10 BH steps"},
            "e2e": {"value": v, "unit": "converged minimisations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_cuda(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import lj_bh as L

    dev = torch.device("cuda", local)
    ctx = L.Ctx(local)
    ctx.reserve(WALKERS * K, N_ATOMS, 10)
    x0, seed = start_state(rank)
    walker0 = rank * WALKERS
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    if args.micro_only:
        if rank == 0:
            print(json.dumps({"eval_microbench": eval_microbench(L, ctx, dev, flush,
                                                                 args.micro_repeats)}), flush=True)
        ctx.close()
        return 0

    def init_state():
        x = torch.as_tensor(x0.reshape(-1), dtype=torch.float64, device=dev).contiguous()
        e = torch.empty(WALKERS, dtype=torch.float64, device=dev)
        st = torch.empty(WALKERS, dtype=torch.int32, device=dev)
        L.lbfgs_minimize_batched(ctx, x, e, st, n_cand=WALKERS, uniform_n=N_ATOMS,
                                 params=L.LbfgsParams(prec=L.LJ_PREC_FP64))
        xm = x.view(WALKERS, -1)
        return {"x_cur": xm.clone(), "e_cur": e.clone(), "x_best": xm.clone(),
                "e_best": e.clone(), "stepsize": torch.full((WALKERS,), STEP0, dtype=torch.float64,
                                                            device=dev),
                "win_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev),
                "n_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev)}

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_run(prec, n_steps, warmup):
        state = init_state()
        p = L.BhParams(K=K, kT=KT, seed=seed, n_steps=BH_PER_LAUNCH, walker0=walker0,
                       min=L.LbfgsParams(prec=prec, switch_gtol=SWITCH_GTOL))
        for s in range(warmup):
            p.step0 = s * BH_PER_LAUNCH
            L.bh_step_batched(ctx, state, p)
        stats = L.new_stats(dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n_steps)]
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            t0 = time.perf_counter()
            for s in range(n_steps):
                flush.fill_(float(s))
                p.step0 = (warmup + s) * BH_PER_LAUNCH
                ev[s][0].record(stream)
                L.bh_step_batched(ctx, state, p, None, stats)
                ev[s][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return sum(ms) / 1e3, wall, L.stats_dict(stats), clk.summary(), state

    def e2e_run(prec, n_steps, warmup):
        """Public API with host buffers: pinned H2D of the walker state, the
        BH step, D2H of the updated state, every step."""
        dstate = init_state()
        host = {k: v.cpu().pin_memory() for k, v in dstate.items()}
        p = L.BhParams(K=K, kT=KT, seed=seed, n_steps=BH_PER_LAUNCH, walker0=walker0,
                       min=L.LbfgsParams(prec=prec, switch_gtol=SWITCH_GTOL))
        stats = L.new_stats(dev)
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        for s in range(warmup + n_steps):
            if s == warmup:
                stats.zero_()
                torch.cuda.synchronize()
                barrier()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            for k in host:
                dstate[k].copy_(host[k], non_blocking=True)
            p.step0 = s * BH_PER_LAUNCH
            L.bh_step_batched(ctx, dstate, p, None, stats)
            for k in host:
                host[k].copy_(dstate[k], non_blocking=True)
            torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        barrier()
        return wall, L.stats_dict(stats), h2d

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64)
        torch.distributed.all_reduce(t)
        return float(t.item())

    # ---- mixed precision (headline) ----------------------------------------
    t_dev, wall, st_mix, clocks, _ = timed_run(L.LJ_PREC_MIXED, args.steps, args.warmup)
    t_dev = max_over_ranks(t_dev)
    conv = sum_over_ranks(st_mix["converged"])
    mins = sum_over_ranks(st_mix["minimisations"])
    value = conv / t_dev
    flops, flops64 = flops_from_stats(st_mix)
    achieved_tf = flops / t_dev / 1e12 if world == 1 else None
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "steps": args.steps, "ms_per_step":
                              1e3 * t_dev / args.steps, "work": st_mix}), flush=True)
        ctx.close()
        return 0
    # ---- FP64 path on the same workload --------------------------------------
    n64 = args.fp64_steps if args.fp64_steps is not None else max(2, args.steps // 10)
    t64, _, st64, _, _ = timed_run(L.LJ_PREC_FP64, n64, min(args.warmup, 3))
    t64 = max_over_ranks(t64)
    value64 = sum_over_ranks(st64["converged"]) / t64
    flops_64path, _ = flops_from_stats(st64)
    # ---- evaluation microbench (pair evals/s) ---------------------------------
    micro = None
    if not args.no_micro and world == 1:
        micro = eval_microbench(L, ctx, dev, flush)
    # ---- end to end -------------------------------------------------------------
    e2e = None
    if not args.no_e2e:
        wall_e2e, st_e2e, h2d = e2e_run(L.LJ_PREC_MIXED, max(3, args.steps // 5),
                                        min(args.warmup, 3))
        wall_e2e = max_over_ranks(wall_e2e)
        e2e = {"value": sum_over_ranks(st_e2e["converged"]) / wall_e2e,
               "unit": "converged minimisations/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d}
    line = {
        "metric": "converged LJ minimisations/s",
        "value": value,
        "unit": "converged minimisations/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * t_dev / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_atoms": N_ATOMS, "walkers_per_gpu": WALKERS, "K": K,
                   "bh_steps_per_step": BH_PER_LAUNCH,
                   "minimisations_per_step": WALKERS * K * BH_PER_LAUNCH * world,
                   "precision": "mixed", "switch_gtol": SWITCH_GTOL,
                   "l2": "flushed (256 MiB write) between timed steps"},
        "minimisations_per_s": mins / t_dev,
        "converged_fraction": conv / max(mins, 1),
        "fp64_path": {"value": value64, "unit": "converged minimisations/s", "steps": n64,
                      "ms_per_step": 1e3 * t64 / n64,
                      "mixed_over_fp64": value / value64 if value64 > 0 else None,
                      "achieved_tflops": flops_64path / t64 / 1e12,
                      "fp64_peak_tflops_nominal": FP64_PEAK_TFLOPS},
        "work": {k: st_mix[k] for k in ("evals32", "evals64", "evals_df", "iters32", "iters64",
                                        "cycles32", "cycles_df", "cycles64", "cycles_direction",
                                        "cycles_linesearch")},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "wall_s_timed_region": wall,
    }
    if achieved_tf is not None:
        line["roofline"] = {"bound": "alu", "achieved": achieved_tf, "peak": FP32_PEAK_TFLOPS,
                            "unit": "TFLOP/s", "frac": achieved_tf / FP32_PEAK_TFLOPS,
                            "traffic": BH_DRAM_BYTES_PER_LAUNCH,
                            "traffic_unit": "DRAM bytes per launch (ncu)",
                            "kernel": "bh_cluster_kernel<64,1,mixed>",
                            "fp64_flop_share": flops64 / flops if flops else None}
    if e2e:
        line["e2e"] = e2e
    if micro:
        line["eval_microbench"] = micro
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(x0, seed)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# other workloads (one GPU): (name, n_cand, N range, start kind, m)
BATCH_WORKLOADS = {
    "uneven-4096": dict(n_cand=4096, n_lo=13, n_hi=150, kind="cube", m=10, cfg=3,
                        desc="4,096 candidates, N uniform in [13, 150], cube starts at "
                             "reduced density 0.3, bucketed persistent launches, m=10"),
    "large-500": dict(n_cand=1024, n_lo=500, n_hi=500, kind="fcc", m=20, cfg=4,
                      desc="1,024 candidates of N=500, fcc fragments jittered 0.1 sigma, m=20"),
    "large-1000": dict(n_cand=256, n_lo=1000, n_hi=1000, kind="fcc", m=20, cfg=4,
                       desc="256 candidates of N=1000, fcc fragments jittered 0.1 sigma, m=20"),
}


def run_batch_workload(args):
    """Batched minimisation of one workload, mixed and FP64, each timed with
    CUDA events around lbfgs_minimize_batched (inputs resident, L2 flushed
    before each timed call); converged minimisations per second."""
    import torch
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import inputs as I
    from paper_2510_25938_gb300 import lj_bh as L
    w = BATCH_WORKLOADS[args.workload]
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    seed = I.workload_seed(w["cfg"])
    if w["kind"] == "cube":
        sizes = I.uneven_sizes(w["n_cand"], w["n_lo"], w["n_hi"], seed)
        x0, off = I.uneven_cube_starts(sizes, 0.3, seed + 1)
        uniform = 0
    else:
        x0 = I.fcc_fragments(w["n_cand"], w["n_lo"], 0.1, seed + w["n_lo"]).reshape(-1)
        off = None
        uniform = w["n_lo"]
    n_cand = w["n_cand"]
    ctx = L.Ctx(0)
    tuned = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    offd = torch.as_tensor(off, device=dev) if off is not None else None
    out = {}
    for prec, name in ((L.LJ_PREC_MIXED, "mixed"), (L.LJ_PREC_FP64, "fp64")):
        # threads per candidate and switch_gtol chosen per size bucket by the library
        # autotuner: on synthetic cube starts for the uneven batch, on a sample of the
        # workload's own starts (copies, before timing) for the uniform ones
        if offd is None:
            xs = torch.as_tensor(x0, dtype=torch.float64, device=dev).contiguous()
            tuned[name] = ctx.autotune_batch(xs, n_cand, uniform, w["m"], prec,
                                             max_sample=n_cand // 4)
        else:
            tuned[name] = ctx.autotune(w["n_hi"], w["m"], prec)
        times, conv = [], 0
        for rep in range(max(args.warmup, 1) + args.steps):
            x = torch.as_tensor(x0, dtype=torch.float64, device=dev).contiguous()
            e = torch.empty(n_cand, dtype=torch.float64, device=dev)
            st = torch.empty(n_cand, dtype=torch.int32, device=dev)
            stats = L.new_stats(dev)
            flush.fill_(float(rep))
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            kw = dict(atom_offset=offd, max_n=w["n_hi"]) if offd is not None else dict(
                uniform_n=uniform)
            ev0.record()
            L.lbfgs_minimize_batched(ctx, x, e, st, None, None, stats, n_cand=n_cand,
                                     params=L.LbfgsParams(prec=prec, m=w["m"]), **kw)
            ev1.record()
            torch.cuda.synchronize()
            if rep >= max(args.warmup, 1):
                times.append(ev0.elapsed_time(ev1) / 1e3)
                sd = L.stats_dict(stats)
                conv = sd["converged"]
        t = sum(times) / len(times)
        mins = max(sd["minimisations"], 1)
        out[name] = {"value": conv / t, "ms_per_batch": 1e3 * t, "converged_fraction": conv / n_cand,
                     "per_minimisation": {k: sd[k] / mins for k in (
                         "evals32", "evals_df", "evals64", "iters32", "iters64", "cycles32",
                         "cycles_df", "cycles64", "cycles_direction", "cycles_linesearch")}}
    line = {"metric": "converged LJ minimisations/s", "value": out["mixed"]["value"],
            "unit": "converged minimisations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": w["desc"], "precision": "mixed",
                                            "l2": "flushed (256 MiB write) before each batch"},
            "mixed": out["mixed"], "fp64_path": out["fp64"],
            "autotuned_per_bucket": tuned,
            "mixed_over_fp64": out["mixed"]["value"] / out["fp64"]["value"]}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_sequential_lj13(args):
    """One FP64 walker of LJ13 (cube side 2.0 sigma, K=1, 200 BH steps in one
    launch, step 0.4 sigma adapted every 10 steps toward 50%, kT=0.8): BH
    steps per second on the GPU and with the oracle on one host core.  This
    is a latency-bound case; the GPU is not expected to win it."""
    import torch
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import inputs as I
    from paper_2510_25938_gb300 import lj_bh as L
    import oracle as O
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    seed = I.workload_seed(0)
    x0 = I.cube_starts(1, 13, 2.0, seed)
    xm, em, _, _, _ = O.lbfgs_batch(x0, 1, uniform_n=13)
    ctx = L.Ctx(0)
    n_steps = 200

    def state():
        x = torch.as_tensor(xm.reshape(1, -1), dtype=torch.float64, device=dev)
        return {"x_cur": x.clone(), "e_cur": torch.as_tensor(em, device=dev),
                "x_best": x.clone(), "e_best": torch.as_tensor(em, device=dev),
                "stepsize": torch.full((1,), 0.4, dtype=torch.float64, device=dev),
                "win_accept": torch.zeros(1, dtype=torch.int32, device=dev),
                "n_accept": torch.zeros(1, dtype=torch.int32, device=dev)}
    p = L.BhParams(K=1, kT=0.8, seed=seed, n_steps=n_steps, min=L.LbfgsParams(prec=L.LJ_PREC_FP64))
    times = []
    for rep in range(max(args.warmup, 1) + args.steps):
        st = state()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        L.bh_step_batched(ctx, st, p)
        ev1.record()
        torch.cuda.synchronize()
        if rep >= max(args.warmup, 1):
            times.append(ev0.elapsed_time(ev1) / 1e3)
    t = sum(times) / len(times)
    ost = {"x_cur": xm.reshape(1, -1).copy(), "e_cur": em.copy(), "x_best": xm.reshape(1, -1).copy(),
           "e_best": em.copy(), "stepsize": np.full(1, 0.4), "win_accept": np.zeros(1, np.int32),
           "n_accept": np.zeros(1, np.int32)}
    t0 = time.perf_counter()
    O.bh_run(ost, O.BhParamsPy(K=1, kT=0.8, seed=seed, n_steps=n_steps))
    t_cpu = time.perf_counter() - t0
    line = {"metric": "BH steps/s", "value": n_steps / t, "unit": "BH steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "LJ13, one walker, K=1, 200 BH steps in one launch, FP64, "
                                   "cube start side 2.0 sigma, kT=0.8, step 0.4 sigma"},
            "ms_per_200_steps": 1e3 * t,
            "cpu_oracle_one_core": {"value": n_steps / t_cpu, "unit": "BH steps/s", "cores": 1}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in BATCH_WORKLOADS:
        return run_batch_workload(args)
    if args.workload == "lj13-seq":
        return run_sequential_lj13(args)
    return run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())
