"""Command-line Basin Hopping on the GPU, the way the paper's driver runs.

    python -m paper_2510_25938_gb300 input.molden [options]

Reads the first geometry of ``input.molden`` (Methodology, "Initial
Structures and Input"), minimises it, then runs Basin Hopping steps with K
candidates per step (Methodology, "Algorithm Overview": perturbation of every
atom within +-step, K parallel minimisations, the lowest candidate to the
Metropolis test, the step size adapted every `interval` steps toward the
target acceptance rate) and appends every accepted structure, with its step
and energy (and the minimiser's status for that candidate), to
``input_accepted.molden`` ("Running the Code").  The defaults
follow the paper: eps = sigma = 1, T = 1.0, 200 steps, adaptation every 10
steps toward 50%, up to eight candidates (K = 8), L-BFGS to ||grad E||_inf <
1e-6.  Every step runs in the library's bh_step_batched kernel (one launch
per step, so that each accepted structure can be written out); there is no
CPU path.  ``--walkers W`` runs W independent chains from the same start
(different random streams) and writes each one's accepted structures to its
own file.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np


STATUS_NAMES = {0: "converged", 1: "maxiter", 2: "linesearch_fail", 3: "nonfinite",
                4: "timeout", 5: "bad_input"}


def parse(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2510_25938_gb300",
                                 description="GPU Basin Hopping of a Lennard-Jones cluster "
                                             "from a Molden file")
    ap.add_argument("input", help="Molden (or XYZ) file; its first geometry is the start")
    ap.add_argument("--steps", type=int, default=200, help="Basin Hopping steps (200)")
    ap.add_argument("--candidates", "-K", type=int, default=8,
                    help="parallel candidates per step (8)")
    ap.add_argument("--kT", type=float, default=1.0, help="Metropolis temperature (1.0)")
    ap.add_argument("--step", type=float, default=0.4,
                    help="initial perturbation half-width in sigma (0.4)")
    ap.add_argument("--interval", type=int, default=10, help="adaptation interval (10)")
    ap.add_argument("--target", type=float, default=0.5, help="target acceptance rate (0.5)")
    ap.add_argument("--factor", type=float, default=0.9, help="adaptation factor (0.9)")
    ap.add_argument("--seed", type=int, default=2510259380, help="Philox seed")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--m", type=int, default=10, help="L-BFGS history length (10)")
    ap.add_argument("--gtol", type=float, default=1e-6, help="||grad E||_inf tolerance (1e-6)")
    ap.add_argument("--walkers", type=int, default=1, help="independent chains (1)")
    ap.add_argument("--output", default=None,
                    help="accepted-structure file (default <input>_accepted.molden; with "
                         "several walkers _w<i> is inserted before the extension)")
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--json", action="store_true", help="print the summary as JSON")
    return ap.parse_args(argv)


def _out_path(args, w):
    from . import molden
    base = args.output or molden.accepted_path(args.input)
    if args.walkers == 1:
        return base
    root, ext = os.path.splitext(base)
    return f"{root}_w{w}{ext}"


def main(argv=None) -> int:
    args = parse(argv)
    import torch
    from . import build as B
    from . import molden
    B.build()
    from . import lj_bh as L
    if not torch.cuda.is_available():
        raise SystemExit("a CUDA device is required (the library has no CPU path)")
    torch.cuda.set_device(args.device)
    dev = torch.device("cuda", args.device)
    g0 = molden.read_first_geometry(args.input)
    n = len(g0.symbols)
    W, K = args.walkers, args.candidates
    prec = L.LJ_PREC_MIXED if args.precision == "mixed" else L.LJ_PREC_FP64
    ctx = L.Ctx(args.device)
    lp = L.LbfgsParams(prec=prec, m=args.m, gtol=args.gtol)
    x = torch.as_tensor(np.tile(g0.flat, W), dtype=torch.float64, device=dev).contiguous()
    e = torch.empty(W, dtype=torch.float64, device=dev)
    st0 = torch.empty(W, dtype=torch.int32, device=dev)
    L.lbfgs_minimize_batched(ctx, x, e, st0, n_cand=W, uniform_n=n, params=lp)
    xm = x.view(W, -1)
    state = {"x_cur": xm.clone(), "e_cur": e.clone(), "x_best": xm.clone(), "e_best": e.clone(),
             "stepsize": torch.full((W,), args.step, dtype=torch.float64, device=dev),
             "win_accept": torch.zeros(W, dtype=torch.int32, device=dev),
             "n_accept": torch.zeros(W, dtype=torch.int32, device=dev)}
    p = L.BhParams(K=K, kT=args.kT, target_rate=args.target, interval=args.interval,
                   factor=args.factor, seed=args.seed, n_steps=1, min=lp)
    tr = L.new_trace(1, W, K, dev)
    e_start = e.cpu().numpy()
    paths = [_out_path(args, w) for w in range(W)]
    for w in range(W):                       # the minimised start opens each file
        molden.write_geometries(paths[w], [molden.Geometry(
            g0.symbols, xm[w].cpu().numpy().reshape(n, 3),
            f"step -1 (minimised start) energy {e_start[w]:.12f}")], append=False)
    accepted_total = np.zeros(W, dtype=np.int64)
    for s in range(args.steps):
        p.step0 = s
        L.bh_step_batched(ctx, state, p, tr)
        acc = tr["accepted"][0].cpu().numpy()
        if acc.any():
            xc = state["x_cur"].cpu().numpy()
            ec = state["e_cur"].cpu().numpy()
            te = tr["trial_e"][0].cpu().numpy()
            ts = tr["trial_status"][0].cpu().numpy()
            for w in np.nonzero(acc)[0]:
                # the selected candidate: the lowest finite energy, ties to the lowest k
                fin = np.where(np.isfinite(te[w]), te[w], np.inf)
                status = STATUS_NAMES.get(int(ts[w, int(np.argmin(fin))]), "unknown")
                molden.write_geometries(paths[w], [molden.Geometry(
                    g0.symbols, xc[w].reshape(n, 3),
                    f"step {s} energy {ec[w]:.12f} status {status}")])
            accepted_total += acc.astype(np.int64)
    torch.cuda.synchronize()
    summary = {"input": args.input, "atoms": n, "walkers": W, "candidates": K,
               "steps": args.steps, "precision": args.precision,
               "start_energy": e_start.tolist(),
               "best_energy": state["e_best"].cpu().numpy().tolist(),
               "final_energy": state["e_cur"].cpu().numpy().tolist(),
               "acceptance_rate": (accepted_total / max(args.steps, 1)).tolist(),
               "final_step": state["stepsize"].cpu().numpy().tolist(),
               "accepted_files": paths}
    ctx.close()
    if args.json:
        print(json.dumps(summary))
    else:
        for w in range(W):
            print(f"walker {w}: start {e_start[w]:.6f}  best {summary['best_energy'][w]:.6f}  "
                  f"acceptance {summary['acceptance_rate'][w]:.2f}  final step "
                  f"{summary['final_step'][w]:.4f}  -> {paths[w]}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
