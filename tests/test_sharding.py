"""Walker sharding (multi-GPU layout) tested on CPU.

Walkers are independent and every random number is drawn from a counter-based
Philox stream keyed by the GLOBAL walker index (walker0 + local index), so a
run split into shards of walkers reproduces the unsharded run exactly; the
only communication is an end-of-run gather of per-walker results.  The same
sharding is what bench.py does under torchrun (rank r runs walkers
r*W .. r*W+W-1).  Checked with the oracle (the GPU kernels take walker0 the
same way), in one process and as two gloo ranks.
"""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2510_25938_gb300 import inputs as I


def _state(x0):
    W, n3 = x0.shape
    xm, em, st, _, _ = O.lbfgs_batch(x0, W, uniform_n=n3 // 3)
    xm = xm.reshape(W, n3)
    return {"x_cur": xm.copy(), "e_cur": em.copy(), "x_best": xm.copy(), "e_best": em.copy(),
            "stepsize": np.full(W, 0.4), "win_accept": np.zeros(W, np.int32),
            "n_accept": np.zeros(W, np.int32)}


def _slice(st, a, b):
    return {k: np.ascontiguousarray(v[a:b]) for k, v in st.items()}


X0 = I.cube_starts(4, 8, 1.8, seed=31)
PARAMS = dict(K=3, kT=0.8, seed=1234, n_steps=12)


def test_shards_reproduce_unsharded_run():
    full = _state(X0)
    tr_full = O.bh_run(full, O.BhParamsPy(**PARAMS))
    base = _state(X0)
    parts = []
    for a, b in ((0, 2), (2, 4)):
        st = _slice(base, a, b)
        tr = O.bh_run(st, O.BhParamsPy(walker0=a, **PARAMS))
        parts.append((st, tr))
    for key in full:
        got = np.concatenate([p[0][key] for p in parts])
        assert np.array_equal(got, full[key]), key
    for key in ("trial_e", "accepted", "stepsize"):
        got = np.concatenate([p[1][key] for p in parts], axis=1)
        assert np.array_equal(got, tr_full[key]), key


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per = X0.shape[0] // world
    st = _slice(_state(X0), rank * per, (rank + 1) * per)
    O.bh_run(st, O.BhParamsPy(walker0=rank * per, **PARAMS))
    # end-of-run gather of per-walker results (the only exchange)
    e = torch.tensor(st["e_best"])
    x = torch.tensor(st["x_best"])
    es = [torch.zeros_like(e) for _ in range(world)]
    xs = [torch.zeros_like(x) for _ in range(world)]
    dist.all_gather(es, e)
    dist.all_gather(xs, x)
    if rank == 0:
        np.save(os.path.join(out_dir, "e_best.npy"), torch.cat(es).numpy())
        np.save(os.path.join(out_dir, "x_best.npy"), torch.cat(xs).numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    full = _state(X0)
    O.bh_run(full, O.BhParamsPy(**PARAMS))
    assert np.array_equal(np.load(tmp_path / "e_best.npy"), full["e_best"])
    assert np.array_equal(np.load(tmp_path / "x_best.npy"), full["x_best"])
