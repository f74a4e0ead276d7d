#!/usr/bin/env python3
"""Benchmark: batched LJ38 Basin Hopping on GB300 (one JSON line on stdout).

Workload: LJ38 (eps = sigma = 1), 64 independent walkers x K = 8 candidates
per BH step (512 local minimisations per BH step), 500 BH steps, starts
uniform in a cube of side 3.2 sigma (seeded), minimised once before timing;
perturbations +-step per coordinate from Philox (initial step 0.4 sigma,
adapted every 10 steps toward 50% acceptance), kT = 0.8, L-BFGS m = 10 to
||grad E||_inf < 1e-6.  One bench "step" is one bh_step_batched launch that
advances every walker by 25 BH steps (12,800 local minimisations); the timed
steps run the workload's BH steps from step 0 (warm-up launches advance a
copy of the state), so the default 20 steps are the workload's 500 BH steps.

metric  converged LJ minimisations per second (minimisations that reached
        ||grad E||_inf < 1e-6 with an FP64 gradient), mixed precision path;
        the FP64 path is measured on the same workload for comparison.
Timing  CUDA events around each step's launch on the launching stream, L2
        flushed (256 MiB write) between steps outside the events; e2e adds,
        every step, the host->device copy of the walker state from pinned
        memory and the device->host copy of the updated state.
N > 1   (torchrun) each rank runs its own 64 walkers (global walker indices
        offset by rank): weak scaling, no collective on the data path.
--impl reference   the FP64 CPU oracle on this host's cores, same workload
        (each reference step is one BH step of the 64 walkers).

The same JSON line also carries (one GPU only):
  eval_microbench   energy+gradient throughput on 65,536 jittered LJ38 minima,
                    FP32 and FP64, with per-evaluation errors against the oracle;
  errors            the mixed and FP64 paths against the FP64 oracle on one BH
                    step's 512 trial moves (identical Philox inputs): same-basin
                    fraction and |dE| on same-basin minima;
  k_sweep           wall-clock per BH step and converged/s for K = 1..16;
  search_quality    running best energy and hits of the LJ38 truncated
                    octahedron over the workload's 500 BH steps (mixed and,
                    as search_quality_fp64, the FP64 path);
  other_workloads   the sequential LJ13 walker, the uneven 4,096-candidate batch
                    (one CUDA-graph replay), the 500- and 1000-atom batches and
                    the same Basin Hopping workload on the Morse potential
                    (rho = 6), mixed and FP64, each with an oracle sample on the
                    host cores.
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
# BH steps per bench step.  A launch ends when the slowest of its 64 walkers
# has finished its steps, so the walkers' spread in time per step costs once
# per launch: on this workload 10 steps per launch took 2.024 ms per BH step,
# 50 took 1.916 (CUDA events, same steps); 25 makes 20 bench steps the
# workload's 500 BH steps
BH_PER_LAUNCH = 25
# BH steps per launch of the search-quality run, which reads the walkers'
# best energies after every launch
SEARCH_PER_LAUNCH = 10
SIDE, STEP0, KT = 3.2, 0.4, 0.8
# MIXED precision policy parameter of this workload: the FP32 tier's gradient
# threshold (swept on LJ38 BH: 1e-3 168k, 3e-4 179k, 1e-4 183k converged/s);
# the bench runs lj_ctx_autotune_bh on the workload first and passes 0
# (automatic: the tuned value) unless --no-tune, which passes this one
SWITCH_GTOL = 1e-4
CONFIG_ID = 1
WORKLOAD = ("LJ38 Basin Hopping: 64 walkers x K=8 candidates per BH step (512 L-BFGS "
            "minimisations per BH step), 25 BH steps per bench step, cube starts side "
            "3.2 sigma, m=10, ||g||_inf<1e-6")
PAIRS = N_ATOMS * (N_ATOMS - 1) // 2
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e-3   # SMs x FP32 lanes x 2 (FMA) x max SM GHz
FP64_PEAK_TFLOPS = 1.25                    # nominal FP64 (non-tensor) rate of GB300
# dram__bytes_read.sum + dram__bytes_write.sum of one bh_cluster_kernel launch of this
# workload (25 BH steps), from one ncu capture of the launch as the bench makes it; None
# whenever the kernel or the launch changes until it is captured again
BH_DRAM_BYTES_PER_LAUNCH = 1097216


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-micro", action="store_true", help="skip the evaluation microbench")
    ap.add_argument("--workload", default="lj38-bh",
                    choices=["lj38-bh", "uneven-4096", "large-500", "large-1000", "lj13-seq",
                             "morse38-bh"],
                    help="lj38-bh (default): the Basin Hopping step this bench reports; the "
                         "others time the batched minimisation of the uneven and large-cluster "
                         "workloads, one sequential FP64 LJ13 walker, or the Basin Hopping "
                         "workload on the Morse potential, and print their own line")
    ap.add_argument("--micro-only", action="store_true",
                    help="run only the evaluation microbench and print its JSON")
    ap.add_argument("--micro-repeats", type=int, default=100)
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (lj_ctx_autotune_bh, or lj_ctx_autotune for the "
                         "batched workloads): library default team and history placement, "
                         "switch_gtol 1e-4")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline, FP64 path and e2e only (no error, K-sweep, search-quality "
                         "or other-workload blocks)")
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


def bh_state_np(xm, em, step0=STEP0):
    W = xm.shape[0]
    return {"x_cur": xm.copy(), "e_cur": em.copy(), "x_best": xm.copy(), "e_best": em.copy(),
            "stepsize": np.full(W, step0), "win_accept": np.zeros(W, np.int32),
            "n_accept": np.zeros(W, np.int32)}


def cpu_baseline(x0, seed, budget_s=12.0):
    """The FP64 oracle on this host's cores: BH steps of all 64 walkers, as
    many as fit in ~budget_s (at least one)."""
    import oracle as O
    xm, em, st, _, _ = O.lbfgs_batch(x0, x0.shape[0], uniform_n=N_ATOMS)
    state = bh_state_np(xm.reshape(x0.shape[0], -1), em)
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


# ---------------------------------------------------------------------------
# error statistics against the oracle (the definitions of the precision
# contract: relative energy error, gradient error against the larger of the
# gradient norm and its no-cancellation scale, same-basin fingerprint)
# ---------------------------------------------------------------------------
SAME_BASIN_TOL = 1e-3


def fingerprint(x):
    """Sorted pair distances: invariant under translation, rotation,
    reflection and permutation; two minima are the same basin when these
    agree to SAME_BASIN_TOL sigma."""
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    d = np.sqrt(((p[:, None, :] - p[None, :, :]) ** 2).sum(-1))
    return np.sort(d[np.triu_indices(len(p), 1)])


def grad_nc_scale(x):
    """||(sum_j |c_ij (x_i - x_j)|)_i||_2: the gradient without cancellation."""
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    d = p[:, None, :] - p[None, :, :]
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    s6 = r2 ** -3
    c = 24.0 * (2 * s6 * s6 - s6) / r2
    return float(np.linalg.norm((np.abs(c)[:, :, None] * np.abs(d)).sum(1)))


def energy_nc_scale(x):
    """4 sum_{i<j} (s12 + s6): the energy without cancellation, the scale a sum
    of rounded pair terms has its error measured against."""
    p = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    d = p[:, None, :] - p[None, :, :]
    r2 = (d ** 2).sum(-1)[np.triu_indices(len(p), 1)]
    s6 = r2 ** -3
    return float(4.0 * (s6 * s6 + s6).sum())


def compare_minima(xg, eg, sg, xo, eo, so, n_atoms):
    """Same-basin fraction among candidates both sides converged, and |dE|
    on the same-basin ones."""
    import oracle as O
    n = eg.size
    xg = xg.reshape(n, -1)
    xo = xo.reshape(n, -1)
    both = same = 0
    de = []
    for c in range(n):
        if sg[c] == O.CONVERGED and so[c] == O.CONVERGED:
            both += 1
            fa, fb = fingerprint(xg[c]), fingerprint(xo[c])
            if np.abs(fa - fb).max() <= SAME_BASIN_TOL:
                same += 1
                de.append(abs(eg[c] - eo[c]))
    de = np.array(de) if de else np.zeros(0)
    return {"candidates": int(n), "both_converged": both, "same_basin": same,
            "same_basin_fraction": same / max(both, 1),
            "max_abs_dE_same_basin": float(de.max()) if de.size else None,
            "median_abs_dE_same_basin": float(np.median(de)) if de.size else None,
            "gpu_converged_fraction": float((sg == O.CONVERGED).mean()),
            "oracle_converged_fraction": float((so == O.CONVERGED).mean())}


def eval_errors(cfg, en32, gr32, en64, gr64, n_sample=4096):
    """Per-evaluation errors of the FP32 and FP64 evaluations against the
    oracle on a sample of the microbench configurations (each side at the
    coordinates it was given: FP32 at the rounded ones)."""
    import oracle as O
    idx = np.linspace(0, cfg.shape[0] - 1, n_sample).astype(np.int64)
    out = {"sample": f"{n_sample} of {cfg.shape[0]} configurations"}
    for name, en, gr, x in (("fp32", en32, gr32, cfg.astype(np.float32).astype(np.float64)),
                            ("fp64", en64, gr64, cfg)):
        xs = x[idx]
        e_ref, g_ref = O.eval_batch(xs, n_sample, uniform_n=N_ATOMS)
        g_ref = g_ref.reshape(n_sample, -1)
        e = en[idx]
        g = gr.reshape(cfg.shape[0], -1)[idx].astype(np.float64)
        rel_e = np.abs(e - e_ref) / np.abs(e_ref)
        gn = np.linalg.norm(g - g_ref, axis=1)
        scale = np.array([max(np.linalg.norm(g_ref[c]), grad_nc_scale(xs[c]))
                          for c in range(n_sample)])
        nc_e = np.array([energy_nc_scale(xs[c]) for c in range(n_sample)])
        out[name] = {"max_rel_E": float(rel_e.max()), "median_rel_E": float(np.median(rel_e)),
                     "p999_rel_E": float(np.quantile(rel_e, 0.999)),
                     "frac_rel_E_above_1e-6": float((rel_e > 1e-6).mean()),
                     "max_rel_E_nc": float((np.abs(e - e_ref) / nc_e).max()),
                     "max_rel_g": float((gn / scale).max()),
                     "max_rel_g_plain": float((gn / np.linalg.norm(g_ref, axis=1)).max())}
    return out


def eval_microbench(L, ctx, dev, flush, repeats=100, errors=True):
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
    res = {}
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
        res[name] = (en.cpu().numpy(), gr.cpu().numpy())
    out["peaks"] = "FP32: 152 SMs x 128 lanes x 2 x 2.07 GHz; FP64: nominal 1.25 TFLOP/s"
    if errors:
        out["errors_vs_oracle"] = eval_errors(cfg, res["fp32"][0], res["fp32"][1],
                                              res["fp64"][0], res["fp64"][1])
    return out


def run_reference(args):
    """The FP64 oracle on this host's cores, timed on the headline workload:
    one reference step is one BH step of all 64 walkers (K = 8), a bounded
    sample of the GPU arm's bench step of BH_PER_LAUNCH BH steps."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    x0, seed = start_state(0)
    import oracle as O
    xm, em, st, _, _ = O.lbfgs_batch(x0, WALKERS, uniform_n=N_ATOMS)
    # warm-up steps advance a copy; the timed steps are the workload's BH
    # steps 0, 1, ... from the minimised starts, as on the GPU arm
    wstate = bh_state_np(xm.reshape(WALKERS, -1), em)
    for s in range(args.warmup):
        O.bh_run(wstate, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=s, n_steps=1))
    state = bh_state_np(xm.reshape(WALKERS, -1), em)
    conv = mins = 0
    t0 = time.perf_counter()
    for s in range(args.steps):
        tr = O.bh_run(state, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=s, n_steps=1))
        conv += int((tr["trial_status"] == O.CONVERGED).sum())
        mins += tr["trial_status"].size
    dt = time.perf_counter() - t0
    v = conv / dt
    line = {"metric": "converged LJ minimisations/s", "value": v,
            "unit": "converged minimisations/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp64",
                       "bh_steps_per_step": 1,
                       "step": f"one BH step of 64 walkers x K=8 (the GPU arm's step is "
                               f"{BH_PER_LAUNCH})"},
            "cpu_baseline": {"value": v, "unit": "converged minimisations/s",
                             "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"{args.steps} BH steps x 64 walkers x K=8 = {mins} "
                                       f"FP64 minimisations ({conv} converged)"},
            "e2e": {"value": v, "unit": "converged minimisations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# other configurations of the workload family (one GPU)
# ---------------------------------------------------------------------------
BATCH_WORKLOADS = {
    "uneven-4096": dict(n_cand=4096, n_lo=13, n_hi=150, kind="cube", m=10, cfg=3,
                        desc="4,096 candidates, N uniform in [13, 150], cube starts at "
                             "reduced density 0.3, bucketed persistent launches replayed as "
                             "one CUDA graph, m=10"),
    "large-500": dict(n_cand=1024, n_lo=500, n_hi=500, kind="fcc", m=20, cfg=4,
                      desc="1,024 candidates of N=500, fcc fragments jittered 0.1 sigma, m=20"),
    "large-1000": dict(n_cand=256, n_lo=1000, n_hi=1000, kind="fcc", m=20, cfg=4,
                       desc="256 candidates of N=1000, fcc fragments jittered 0.1 sigma, m=20"),
}

# the library keeps a team's L-BFGS history in shared memory while it fits
# (about 100 KB per CTA), else in global memory; these workloads' history
# placement in the mixed (FP32 history) and FP64 paths
HISTORY_OFF_CHIP = {"uneven-4096": False, "large-500": True, "large-1000": True}


def batch_inputs(name):
    from paper_2510_25938_gb300 import inputs as I
    w = BATCH_WORKLOADS[name]
    seed = I.workload_seed(w["cfg"])
    if w["kind"] == "cube":
        sizes = I.uneven_sizes(w["n_cand"], w["n_lo"], w["n_hi"], seed)
        x0, off = I.uneven_cube_starts(sizes, 0.3, seed + 1)
        return x0, off, 0
    x0 = I.fcc_fragments(w["n_cand"], w["n_lo"], 0.1, seed + w["n_lo"]).reshape(-1)
    return x0, None, w["n_lo"]


def batch_cpu_baseline(name, x0, off, uniform, budget_s):
    """The FP64 oracle on the host cores on the first candidates of the
    batch, in chunks until ~budget_s."""
    import oracle as O
    w = BATCH_WORKLOADS[name]
    n_total = w["n_cand"]
    chunk = 4 * max(1, O.num_threads())
    done = conv = 0
    t0 = time.perf_counter()
    while done < n_total and (done == 0 or time.perf_counter() - t0 < budget_s):
        c1 = min(n_total, done + chunk)
        if uniform:
            xs = x0[3 * uniform * done:3 * uniform * c1]
            _, _, st, _, _ = O.lbfgs_batch(xs, c1 - done, uniform_n=uniform,
                                           params=O.MinParams(m=w["m"]))
        else:
            sub = off[done:c1 + 1] - off[done]
            xs = x0[3 * off[done]:3 * off[c1]]
            _, _, st, _, _ = O.lbfgs_batch(xs, c1 - done, atom_off=sub,
                                           params=O.MinParams(m=w["m"]))
        conv += int((st == O.CONVERGED).sum())
        done = c1
    dt = time.perf_counter() - t0
    return {"value": conv / dt, "unit": "converged minimisations/s", "cores": O.num_threads(),
            "kind": "oracle",
            "sample": f"first {done} of {n_total} candidates ({conv} converged) in {dt:.1f} s"}


# switch_gtol the autotuner picks for the fcc-fragment workloads (and the
# value the batched workloads use when run without the autotuner)
BATCH_SWITCH_GTOL_UNTUNED = 1e-4


def time_batch(L, ctx, name, prec, x0, off, uniform, reps, warmup, flush, graph, tune=True):
    """Batched minimisation of one workload, autotuned (unless tune is False:
    default team sizes, switch_gtol 1e-4), timed with CUDA events around each
    call (or each replay of one captured CUDA graph of the call), inputs
    resident and L2 flushed before each timed call."""
    import torch
    w = BATCH_WORKLOADS[name]
    dev = torch.device("cuda", torch.cuda.current_device())
    n_cand = w["n_cand"]
    xin = torch.as_tensor(x0, dtype=torch.float64, device=dev).contiguous()
    offd = torch.as_tensor(off, device=dev) if off is not None else None
    if not tune:
        tuned = None
    elif offd is None:
        tuned = ctx.autotune_batch(xin, n_cand, uniform, w["m"], prec, max_sample=n_cand // 4)
    else:
        tuned = ctx.autotune(w["n_hi"], w["m"], prec)
    ctx.reserve(n_cand, w["n_hi"], w["m"])
    x = xin.clone()
    e = torch.empty(n_cand, dtype=torch.float64, device=dev)
    st = torch.empty(n_cand, dtype=torch.int32, device=dev)
    stats = L.new_stats(dev)
    kw = dict(atom_offset=offd, max_n=w["n_hi"]) if offd is not None else dict(uniform_n=uniform)
    p = L.LbfgsParams(prec=prec, m=w["m"],
                      switch_gtol=0.0 if tune else BATCH_SWITCH_GTOL_UNTUNED)

    def call():
        L.lbfgs_minimize_batched(ctx, x, e, st, None, None, stats, n_cand=n_cand, params=p, **kw)

    g = None
    if graph:
        call()                                   # eager call before capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            call()
    times, sd = [], None
    for rep in range(max(warmup, 1) + reps):
        x.copy_(xin)
        stats.zero_()
        flush.fill_(float(rep))
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        if g is not None:
            g.replay()
        else:
            call()
        ev1.record()
        torch.cuda.synchronize()
        if rep >= max(warmup, 1):
            times.append(ev0.elapsed_time(ev1) / 1e3)
            sd = L.stats_dict(stats)
    t = sum(times) / len(times)
    mins = max(sd["minimisations"], 1)
    n_atoms_total = int(off[-1]) if off is not None else n_cand * uniform
    b = 4 if prec == L.LJ_PREC_MIXED else 8
    io_bytes = 48 * n_atoms_total + 16 * n_cand          # x in and out (FP64), energy, status
    hist_bytes = 0
    if HISTORY_OFF_CHIP[name]:
        # two-loop recursion: s_i and y_i read in each loop, the new pair written
        hist_bytes = 4 * b * (sd["vec_elems32"] + sd["vec_elems64"]) + \
            2 * b * 3 * uniform * (sd["iters32"] + sd["iters64"])
    out = {"value": sd["converged"] / t, "unit": "converged minimisations/s",
           "ms_per_batch": 1e3 * t, "converged_fraction": sd["converged"] / n_cand,
           "timed_calls": len(times), "graph_replay": g is not None,
           "hbm_gbs_algorithmic": (io_bytes + hist_bytes) / t / 1e9,
           "history_off_chip": HISTORY_OFF_CHIP[name],
           "autotuned": tuned,
           "per_minimisation": {k: sd[k] / mins for k in (
               "evals32", "evals_df", "evals64", "iters32", "iters64", "cycles32",
               "cycles_df", "cycles64", "cycles_direction", "cycles_linesearch")}}
    if hist_bytes:
        out["history_gbs_algorithmic"] = hist_bytes / t / 1e9
    return out


def batch_workload_record(L, name, flush, reps, warmup, cpu_budget, tune=True):
    w = BATCH_WORKLOADS[name]
    x0, off, uniform = batch_inputs(name)
    rec = {"workload": w["desc"]}
    for prec, pname in ((L.LJ_PREC_MIXED, "mixed"), (L.LJ_PREC_FP64, "fp64")):
        ctx = L.Ctx()
        rec[pname] = time_batch(L, ctx, name, prec, x0, off, uniform,
                                reps if pname == "mixed" else max(1, reps // 2), warmup, flush,
                                graph=(off is not None), tune=tune)
        ctx.close()
    rec["value"] = rec["mixed"]["value"]
    rec["mixed_over_fp64"] = rec["mixed"]["value"] / max(rec["fp64"]["value"], 1e-30)
    if cpu_budget > 0:
        rec["cpu_baseline"] = batch_cpu_baseline(name, x0, off, uniform, cpu_budget)
    return rec


def run_batch_workload(args):
    """--workload uneven-4096 | large-500 | large-1000: one line for that
    configuration alone."""
    import torch
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import lj_bh as L
    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rec = batch_workload_record(L, args.workload, flush, args.steps, args.warmup,
                                0.0 if args.no_cpu_baseline else 10.0, tune=not args.no_tune)
    line = {"metric": "converged LJ minimisations/s", "value": rec["value"],
            "unit": "converged minimisations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": rec["workload"], "precision": "mixed",
                                            "l2": "flushed (256 MiB write) before each batch"}}
    line.update({k: v for k, v in rec.items() if k not in ("workload", "value")})
    print(json.dumps(line), flush=True)
    return 0


def sequential_lj13_record(L, reps, warmup):
    """One FP64 walker of LJ13 (cube side 2.0 sigma, K=1, 200 BH steps in one
    launch, step 0.4 sigma adapted every 10 steps toward 50%, kT=0.8): BH
    steps per second on the GPU and with the oracle on one host core.  This
    is a latency-bound case; the GPU is not expected to win it."""
    import torch
    from paper_2510_25938_gb300 import inputs as I
    import oracle as O
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = I.workload_seed(0)
    x0 = I.cube_starts(1, 13, 2.0, seed)
    xm, em, _, _, _ = O.lbfgs_batch(x0, 1, uniform_n=13)
    ctx = L.Ctx()
    n_steps = 200

    def state():
        x = torch.as_tensor(xm.reshape(1, -1), dtype=torch.float64, device=dev)
        return {"x_cur": x.clone(), "e_cur": torch.as_tensor(em, device=dev),
                "x_best": x.clone(), "e_best": torch.as_tensor(em, device=dev),
                "stepsize": torch.full((1,), 0.4, dtype=torch.float64, device=dev),
                "win_accept": torch.zeros(1, dtype=torch.int32, device=dev),
                "n_accept": torch.zeros(1, dtype=torch.int32, device=dev)}
    out = {"workload": "LJ13, one walker, K=1, 200 BH steps in one launch, cube start side "
                       "2.0 sigma, kT=0.8, step 0.4 sigma"}
    for prec, pname in ((L.LJ_PREC_FP64, "fp64"), (L.LJ_PREC_MIXED, "mixed")):
        p = L.BhParams(K=1, kT=0.8, seed=seed, n_steps=n_steps, min=L.LbfgsParams(prec=prec))
        times, conv = [], 0
        for rep in range(max(warmup, 1) + reps):
            st = state()
            stats = L.new_stats(dev)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            L.bh_step_batched(ctx, st, p, None, stats)
            ev1.record()
            torch.cuda.synchronize()
            if rep >= max(warmup, 1):
                times.append(ev0.elapsed_time(ev1) / 1e3)
                sd = L.stats_dict(stats)
                conv = sd["converged"]
        t = sum(times) / len(times)
        out[pname] = {"bh_steps_per_s": n_steps / t, "ms_per_200_steps": 1e3 * t,
                      "value": conv / t, "unit": "converged minimisations/s",
                      "per_minimisation": {k: sd[k] / max(sd["minimisations"], 1) for k in (
                          "evals32", "evals_df", "evals64", "iters32", "iters64", "cycles32",
                          "cycles_df", "cycles64", "cycles_direction", "cycles_linesearch")}}
    ctx.close()
    ost = bh_state_np(xm.reshape(1, -1), em, 0.4)
    t0 = time.perf_counter()
    tro = O.bh_run(ost, O.BhParamsPy(K=1, kT=0.8, seed=seed, n_steps=n_steps), n_threads=1)
    t_cpu = time.perf_counter() - t0
    conv = int((tro["trial_status"] == O.CONVERGED).sum())
    out["value"] = out["fp64"]["value"]
    out["cpu_baseline"] = {"value": conv / t_cpu, "unit": "converged minimisations/s",
                           "bh_steps_per_s": n_steps / t_cpu, "cores": 1, "kind": "oracle",
                           "sample": "the same 200 FP64 BH steps on one core"}
    return out


def run_sequential_lj13(args):
    import torch
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import lj_bh as L
    torch.cuda.set_device(0)
    rec = sequential_lj13_record(L, args.steps, args.warmup)
    line = {"metric": "BH steps/s", "value": rec["fp64"]["bh_steps_per_s"], "unit": "BH steps/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "dtype": "f64", "data": "synthetic", "config": {"workload": rec["workload"]}}
    line.update({k: v for k, v in rec.items() if k != "workload"})
    print(json.dumps(line), flush=True)
    return 0


# Morse pair potential (the pair-potential extension of the method): the
# headline's Basin Hopping workload with Eq. (1) replaced by Morse, rho = 6
MORSE_RHO = 6.0
# algorithmic flops of one Morse pair (difference 3, r^2 5, r 1, exponent 2,
# exp 1, e(e-2) 2, e(e-1)/r 3, three gradient products and sums 6, energy
# sum 1, counting the square root and the exponential as one each)
MORSE_PAIR_FLOPS = 24.0


def morse_bh_record(L, flush, reps, warmup, cpu_budget):
    """Morse clusters of 38 atoms (rho = 6), 64 walkers x K = 8, 25 BH steps
    per launch, cube starts side 3.2 re, kT = 0.8: converged minimisations per
    second, mixed and FP64, with the oracle's Morse on the host cores."""
    import torch
    from paper_2510_25938_gb300 import inputs as I
    import oracle as O
    dev = torch.device("cuda", torch.cuda.current_device())
    seed = I.workload_seed(CONFIG_ID) + 770
    x0 = I.cube_starts(WALKERS, N_ATOMS, SIDE, seed)
    ctx = L.Ctx()
    ctx.reserve(WALKERS * K, N_ATOMS, 10)
    xs = torch.as_tensor(x0.reshape(-1), dtype=torch.float64, device=dev).contiguous()
    es = torch.empty(WALKERS, dtype=torch.float64, device=dev)
    L.lbfgs_minimize_batched(ctx, xs, es, n_cand=WALKERS, uniform_n=N_ATOMS,
                             params=L.LbfgsParams(prec=L.LJ_PREC_FP64, potential=L.LJ_POT_MORSE,
                                                  rho=MORSE_RHO))
    xm = xs.view(WALKERS, -1)

    def state():
        return {"x_cur": xm.clone(), "e_cur": es.clone(), "x_best": xm.clone(),
                "e_best": es.clone(),
                "stepsize": torch.full((WALKERS,), STEP0, dtype=torch.float64, device=dev),
                "win_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev),
                "n_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev)}
    out = {"workload": "Morse rho=6, N=38: 64 walkers x K=8, 25 BH steps per launch, cube "
                       "starts side 3.2 re, kT=0.8, m=10, ||g||_inf<1e-6"}
    for prec, pname in ((L.LJ_PREC_MIXED, "mixed"), (L.LJ_PREC_FP64, "fp64")):
        p = L.BhParams(K=K, kT=KT, seed=seed, n_steps=BH_PER_LAUNCH,
                       min=L.LbfgsParams(prec=prec, switch_gtol=SWITCH_GTOL,
                                         potential=L.LJ_POT_MORSE, rho=MORSE_RHO))
        st = state()
        stats = L.new_stats(dev)
        times = []
        n_rep = reps if pname == "mixed" else max(1, reps // 2)
        for r in range(max(warmup, 1) + n_rep):
            p.step0 = r * BH_PER_LAUNCH
            if r == max(warmup, 1):
                stats.zero_()
            flush.fill_(float(r))
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            L.bh_step_batched(ctx, st, p, None, stats)
            ev1.record()
            torch.cuda.synchronize()
            if r >= max(warmup, 1):
                times.append(ev0.elapsed_time(ev1) / 1e3)
        t = sum(times)
        sd = L.stats_dict(stats)
        fl = MORSE_PAIR_FLOPS * (sd["pairs32"] + sd["pairs64"] + sd["pairs_df"]) + 8.0 * (
            sd["vec_elems32"] + sd["vec_elems64"]) + 12.0 * 3 * N_ATOMS * (
            sd["iters32"] + sd["iters64"])
        out[pname] = {"value": sd["converged"] / t, "unit": "converged minimisations/s",
                      "ms_per_launch": 1e3 * t / len(times), "launches": len(times),
                      "converged_fraction": sd["converged"] / max(sd["minimisations"], 1),
                      "achieved_tflops": fl / t / 1e12,
                      "fp64_pair_share": sd["pairs64"] / max(
                          sd["pairs32"] + sd["pairs64"] + sd["pairs_df"], 1),
                      "per_minimisation": {k: sd[k] / max(sd["minimisations"], 1) for k in (
                          "evals32", "evals_df", "evals64", "iters32", "iters64")}}
    ctx.close()
    out["value"] = out["mixed"]["value"]
    out["mixed_over_fp64"] = out["mixed"]["value"] / max(out["fp64"]["value"], 1e-30)
    out["roofline"] = {"bound": "alu", "achieved": out["mixed"]["achieved_tflops"],
                       "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": out["mixed"]["achieved_tflops"] / FP32_PEAK_TFLOPS,
                       "kernel": "bh_cluster_kernel<64,1,mixed,Morse>",
                       "flops": f"{MORSE_PAIR_FLOPS:g} per pair per evaluation + 8 per history "
                                "element + 36 N per iteration"}
    if cpu_budget > 0:
        em = es.cpu().numpy()
        ost = bh_state_np(xm.cpu().numpy(), em)
        conv = steps = 0
        t0 = time.perf_counter()
        while steps == 0 or time.perf_counter() - t0 < cpu_budget:
            tr = O.bh_run(ost, O.BhParamsPy(K=K, kT=KT, seed=seed, step0=steps, n_steps=1,
                                            potential=O.OBJ_MORSE, rho=MORSE_RHO))
            conv += int((tr["trial_status"] == O.CONVERGED).sum())
            steps += 1
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": conv / dt, "unit": "converged minimisations/s",
                               "cores": O.num_threads(), "kind": "oracle",
                               "sample": f"{steps} FP64 BH steps x 64 walkers x K=8 of Morse38 "
                                         f"({conv} converged) in {dt:.1f} s"}
    return out


def run_morse(args):
    import torch
    from paper_2510_25938_gb300 import build as B
    B.build()
    from paper_2510_25938_gb300 import lj_bh as L
    torch.cuda.set_device(0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    rec = morse_bh_record(L, flush, args.steps, args.warmup,
                          0.0 if args.no_cpu_baseline else 10.0)
    line = {"metric": "converged Morse minimisations/s", "value": rec["value"],
            "unit": "converged minimisations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": rec["workload"], "precision": "mixed",
                                            "l2": "flushed (256 MiB write) before each launch"}}
    line.update({k: v for k, v in rec.items() if k not in ("workload", "value")})
    print(json.dumps(line), flush=True)
    return 0


# LJ38 global minimum: the fcc truncated octahedron (O_h), the structure the
# paper's Results name, minimised by the oracle (stored fixture)
def lj38_global_minimum_energy():
    with open(os.path.join(ROOT, "tests", "golden", "lj38_oh_truncated_octahedron.txt")) as f:
        for line in f:
            if line.startswith("energy"):
                return float(line.split()[1])
    raise RuntimeError("LJ38 reference energy missing")


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

    x_start = torch.as_tensor(x0.reshape(-1), dtype=torch.float64, device=dev).contiguous()
    e_start = torch.empty(WALKERS, dtype=torch.float64, device=dev)
    L.lbfgs_minimize_batched(ctx, x_start, e_start, n_cand=WALKERS, uniform_n=N_ATOMS,
                             params=L.LbfgsParams(prec=L.LJ_PREC_FP64))
    xm_start = x_start.view(WALKERS, -1)

    def init_state():
        return {"x_cur": xm_start.clone(), "e_cur": e_start.clone(), "x_best": xm_start.clone(),
                "e_best": e_start.clone(),
                "stepsize": torch.full((WALKERS,), STEP0, dtype=torch.float64, device=dev),
                "win_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev),
                "n_accept": torch.zeros(WALKERS, dtype=torch.int32, device=dev)}

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def bh_params(prec, k=K, sg=SWITCH_GTOL):
        return L.BhParams(K=k, kT=KT, seed=seed, n_steps=BH_PER_LAUNCH, walker0=walker0,
                          min=L.LbfgsParams(prec=prec, switch_gtol=sg))

    # the library's autotuner picks the BH team, switch_gtol and history
    # placement on copies of this workload's walkers (untimed set-up)
    tuned = None
    sg_run = SWITCH_GTOL
    if not args.no_tune and not args.profile:
        tuned = ctx.autotune_bh(init_state(), bh_params(L.LJ_PREC_MIXED, sg=0.0))
        sg_run = 0.0

    def timed_run(prec, n_steps, warmup):
        # warm-up launches advance a copy; the timed launches run the
        # workload's BH steps 0, 1, ... from the minimised starts
        wstate = init_state()
        p = bh_params(prec, sg=sg_run)
        for s in range(warmup):
            p.step0 = s * BH_PER_LAUNCH
            L.bh_step_batched(ctx, wstate, p)
        state = init_state()
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
                p.step0 = s * BH_PER_LAUNCH
                ev[s][0].record(stream)
                L.bh_step_batched(ctx, state, p, None, stats)
                ev[s][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return sum(ms) / 1e3, wall, L.stats_dict(stats), clk.summary(), state

    def e2e_run(prec, n_steps, warmup):
        """Public API with host buffers, the same steps and L2 flushes as the
        device-timed run: every step copies the walker state from pinned host
        memory to the device, runs the BH launch and copies the updated state
        back, all between the step's CUDA events.  As in timed_run, the timed
        steps start again from the minimised starts at BH step 0."""
        dstate = init_state()
        host0 = {k: v.cpu() for k, v in dstate.items()}
        host = {k: v.clone().pin_memory() for k, v in host0.items()}
        p = bh_params(prec, sg=sg_run)
        stats = L.new_stats(dev)
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(n_steps)]
        for s in range(warmup + n_steps):
            if s == warmup:
                for k in host:
                    host[k].copy_(host0[k])
                stats.zero_()
                torch.cuda.synchronize()
                barrier()
                torch.cuda.synchronize()
            flush.fill_(float(s))
            if s >= warmup:
                ev[s - warmup][0].record(stream)
            for k in host:
                dstate[k].copy_(host[k], non_blocking=True)
            p.step0 = (s if s < warmup else s - warmup) * BH_PER_LAUNCH
            L.bh_step_batched(ctx, dstate, p, None, stats)
            for k in host:
                host[k].copy_(dstate[k], non_blocking=True)
            if s >= warmup:
                ev[s - warmup][1].record(stream)
            torch.cuda.synchronize()
        barrier()
        t = sum(a.elapsed_time(b) for a, b in ev) / 1e3
        return t, L.stats_dict(stats), h2d

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
    t_dev, wall, st_mix, clocks, state_end = timed_run(L.LJ_PREC_MIXED, args.steps, args.warmup)
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
    # ---- end to end: same steps, same flushes, host copies inside the events --
    e2e = None
    if not args.no_e2e:
        t_e2e, st_e2e, h2d = e2e_run(L.LJ_PREC_MIXED, args.steps, args.warmup)
        t_e2e = max_over_ranks(t_e2e)
        e2e = {"value": sum_over_ranks(st_e2e["converged"]) / t_e2e,
               "unit": "converged minimisations/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d, "ms_per_step": 1e3 * t_e2e / args.steps,
               "steps": args.steps,
               "timing": "CUDA events around H2D copies + launch + D2H copies of each "
                         "step, L2 flushed between steps outside the events"}
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
                   "precision": "mixed",
                   "switch_gtol": tuned["switch_gtol"] if tuned else SWITCH_GTOL,
                   "autotuned": ({"team": tuned["team"], "switch_gtol": tuned["switch_gtol"],
                                  "history_global": tuned["history_global"]}
                                 if tuned else None),
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
                            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz "
                                         "(the measured peaks hold no FP32 non-tensor figure)",
                            "fp64_flop_share": flops64 / flops if flops else None}
    if e2e:
        line["e2e"] = e2e
    if world == 1 and not args.no_extras:
        # ---- errors of the timed workload against the oracle ------------------
        line["errors"] = trial_move_errors(L, ctx, dev, state_end, seed,
                                           args.steps * BH_PER_LAUNCH)
        if not args.no_micro:
            line["eval_microbench"] = eval_microbench(L, ctx, dev, flush)
        line["k_sweep"] = k_sweep(L, dev, init_state, bh_params, flush)
        line["search_quality"] = search_quality(L, ctx, dev, init_state, bh_params)
        line["search_quality_fp64"] = search_quality(L, ctx, dev, init_state, bh_params,
                                                     prec=L.LJ_PREC_FP64)
        cpu_b = 0.0 if args.no_cpu_baseline else 5.0
        others = {"lj13-seq": sequential_lj13_record(L, 3, 1)}
        for name in BATCH_WORKLOADS:
            others[name] = batch_workload_record(L, name, flush, 3, 1, cpu_b)
        others["morse38-bh"] = morse_bh_record(L, flush, 3, 1, cpu_b)
        line["other_workloads"] = others
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(x0, seed)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def trial_move_errors(L, ctx, dev, state, seed, step):
    """The trial moves of one BH step of every walker (from the state the
    timed run ended in, perturbed by the oracle's Philox stream, bit-identical
    to the GPU's), minimised by the mixed and the FP64 GPU paths (the
    minimiser the BH kernel runs, through lbfgs_minimize_batched) and by the
    FP64 oracle: same-basin fraction and |dE| on same-basin minima."""
    import torch
    import oracle as O
    xc = state["x_cur"].cpu().numpy()
    step_w = state["stepsize"].cpu().numpy()
    W = xc.shape[0]
    trial = np.stack([O.perturb(xc[w], step_w[w], seed, k, step, w)
                      for w in range(W) for k in range(K)])
    n = trial.shape[0]
    xo, eo, so, _, _ = O.lbfgs_batch(trial, n, uniform_n=N_ATOMS)
    out = {"sample": f"BH step {step}: {W} walkers x K={K} = {n} trial moves of LJ38 from the "
                     f"state the timed run ended in, minimised by the GPU paths and the oracle",
           "same_basin": f"sorted pair distances within {SAME_BASIN_TOL} sigma"}
    for prec, name in ((L.LJ_PREC_MIXED, "mixed"), (L.LJ_PREC_FP64, "fp64")):
        x = torch.as_tensor(trial.reshape(-1), dtype=torch.float64, device=dev).contiguous()
        e = torch.empty(n, dtype=torch.float64, device=dev)
        st = torch.empty(n, dtype=torch.int32, device=dev)
        L.lbfgs_minimize_batched(ctx, x, e, st, n_cand=n, uniform_n=N_ATOMS,
                                 params=L.LbfgsParams(prec=prec, switch_gtol=SWITCH_GTOL))
        torch.cuda.synchronize()
        out[name] = compare_minima(x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy(),
                                   xo, eo, so, N_ATOMS)
    return out


def k_sweep(L, dev, init_state, bh_params, flush, ks=(1, 2, 4, 8, 16), launches=3):
    """Wall-clock per BH step and converged minimisations per second for K
    candidates per walker and step at 64 walkers (the GPU analogue of the
    paper's cumulative wall-clock and speedup against the number of
    concurrent candidates), mixed precision, from the same minimised starts."""
    import torch
    ctx = L.Ctx()
    out = {}
    for k in ks:
        state = init_state()
        p = bh_params(L.LJ_PREC_MIXED, k)
        p.step0 = 0
        L.bh_step_batched(ctx, state, p)          # warm-up launch
        stats = L.new_stats(dev)
        t = 0.0
        for s in range(launches):
            flush.fill_(float(s))
            p.step0 = (s + 1) * BH_PER_LAUNCH
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            L.bh_step_batched(ctx, state, p, None, stats)
            ev1.record()
            torch.cuda.synchronize()
            t += ev0.elapsed_time(ev1) / 1e3
        sd = L.stats_dict(stats)
        out[str(k)] = {"ms_per_bh_step": 1e3 * t / (launches * BH_PER_LAUNCH),
                       "converged_per_s": sd["converged"] / t,
                       "minimisations_per_s": sd["minimisations"] / t}
    base = out[str(ks[0])]["ms_per_bh_step"]
    for k in ks:
        r = out[str(k)]
        # candidates examined per unit time relative to K = 1 (the paper's speedup)
        r["speedup_vs_k1"] = k * base / r["ms_per_bh_step"]
        r["efficiency"] = r["speedup_vs_k1"] / k
    ctx.close()
    return {"walkers": WALKERS, "bh_steps_timed": launches * BH_PER_LAUNCH,
            "precision": "mixed", "per_K": out}


def search_quality(L, ctx, dev, init_state, bh_params, launches=500 // SEARCH_PER_LAUNCH,
                   prec=None):
    """The workload's 500 BH steps from its minimised starts (64 walkers,
    K = 8, mixed unless prec says otherwise): the running best energy against
    BH step, and how many walkers reach the LJ38 global minimum (the O_h
    truncated octahedron)."""
    import torch
    e_gm = lj38_global_minimum_energy()
    state = init_state()
    p = bh_params(L.LJ_PREC_MIXED if prec is None else prec)
    p.n_steps = SEARCH_PER_LAUNCH
    host = torch.empty((launches, WALKERS), dtype=torch.float64).pin_memory()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(launches)]
    for s in range(launches):
        p.step0 = s * SEARCH_PER_LAUNCH
        ev[s][0].record()
        L.bh_step_batched(ctx, state, p)
        ev[s][1].record()
        host[s].copy_(state["e_best"], non_blocking=True)
    torch.cuda.synchronize()
    best = host.numpy().copy()
    ms = np.cumsum([a.elapsed_time(b) for a, b in ev])
    hit = best <= e_gm + 1e-6
    first = np.where(hit.any(0), hit.argmax(0), -1)
    hit_steps = (first[first >= 0] + 1) * SEARCH_PER_LAUNCH
    hit_ms = ms[first[first >= 0]] if (first >= 0).any() else np.zeros(0)
    marks = [s for s in (10, 50, 100, 200, 300, 500) if s <= launches * SEARCH_PER_LAUNCH]
    curve = {str(s): {"lowest": float(best[s // SEARCH_PER_LAUNCH - 1].min()),
                      "mean_of_walker_best": float(best[s // SEARCH_PER_LAUNCH - 1].mean())}
             for s in marks}
    frac = {str(s): float(hit[s // SEARCH_PER_LAUNCH - 1].mean()) for s in marks}
    return {"target": {"energy": e_gm, "structure": "fcc truncated octahedron (O_h)",
                       "tolerance": 1e-6},
            "precision": "mixed" if prec in (None, L.LJ_PREC_MIXED) else "fp64",
            "bh_steps": launches * SEARCH_PER_LAUNCH, "walkers": WALKERS, "K": K,
            "running_best": curve, "fraction_of_walkers_at_target": frac,
            "walkers_hit": int((first >= 0).sum()),
            "median_steps_to_hit": float(np.median(hit_steps)) if hit_steps.size else None,
            "median_gpu_ms_to_hit": float(np.median(hit_ms)) if hit_ms.size else None,
            "gpu_ms_total": float(ms[-1])}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in BATCH_WORKLOADS:
        return run_batch_workload(args)
    if args.workload == "lj13-seq":
        return run_sequential_lj13(args)
    if args.workload == "morse38-bh":
        return run_morse(args)
    return run_cuda(args)


if __name__ == "__main__":
    sys.exit(main())
