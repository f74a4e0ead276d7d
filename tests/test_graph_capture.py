"""CUDA-graph capture of the context entry points.

After lj_ctx_reserve a call within the reserved sizes allocates nothing, so
it can be captured into a CUDA graph: the uneven batch (device-side size
buckets, one persistent launch per bucket) then replays as a single graph
launch, and so does a multi-step Basin Hopping launch.  Replays must give
bit-identical results to eager calls on the same inputs (every candidate is
minimised by one team with the same code, whichever team takes it).
"""
import numpy as np
import pytest

from paper_2510_25938_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lj():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25938_gb300 import build
    build.build()
    from paper_2510_25938_gb300 import lj_bh
    torch.cuda.set_device(0)
    return lj_bh


@pytest.mark.parametrize("prec", [0, 2])
def test_uneven_batch_graph_replay(lj, prec):
    n_cand = 600
    sizes = I.uneven_sizes(n_cand, 13, 150, I.workload_seed(3) + 11)
    x0, off = I.uneven_cube_starts(sizes, 0.3, I.workload_seed(3) + 12)
    x1, _ = I.uneven_cube_starts(sizes, 0.3, I.workload_seed(3) + 13)
    ctx = lj.Ctx(0)
    ctx.reserve(n_cand, int(sizes.max()), 10)
    offd = torch.as_tensor(off, device="cuda")
    p = lj.LbfgsParams(prec=prec)

    def eager(xs):
        x = torch.as_tensor(xs, dtype=torch.float64, device="cuda").contiguous()
        e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
        st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
        lj.lbfgs_minimize_batched(ctx, x, e, st, n_cand=n_cand, atom_offset=offd,
                                  max_n=int(sizes.max()), params=p)
        torch.cuda.synchronize()
        return x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()

    ref0, ref1 = eager(x0), eager(x1)
    xs = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
    es = torch.empty(n_cand, dtype=torch.float64, device="cuda")
    ss = torch.empty(n_cand, dtype=torch.int32, device="cuda")
    stats = lj.new_stats("cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lj.lbfgs_minimize_batched(ctx, xs, es, ss, None, None, stats, n_cand=n_cand,
                                  atom_offset=offd, max_n=int(sizes.max()), params=p)
    for xin, ref in ((x0, ref0), (x1, ref1), (x0, ref0)):
        xs.copy_(torch.as_tensor(xin, dtype=torch.float64, device="cuda"))
        stats.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(xs.cpu().numpy(), ref[0])
        assert np.array_equal(es.cpu().numpy(), ref[1], equal_nan=True)
        assert np.array_equal(ss.cpu().numpy(), ref[2])
        assert lj.stats_dict(stats)["minimisations"] == n_cand
    ctx.close()


def test_bh_steps_graph_replay(lj):
    W, K, N = 16, 4, 38
    seed = I.workload_seed(1) + 21
    x0 = I.cube_starts(W, N, 3.2, seed)
    ctx = lj.Ctx(0)
    ctx.reserve(W * K, N, 10)
    x = torch.as_tensor(x0.reshape(-1), dtype=torch.float64, device="cuda").contiguous()
    e = torch.empty(W, dtype=torch.float64, device="cuda")
    lj.lbfgs_minimize_batched(ctx, x, e, n_cand=W, uniform_n=N,
                              params=lj.LbfgsParams(prec=0))
    torch.cuda.synchronize()
    xm = x.view(W, -1).clone()

    def fresh():
        return {"x_cur": xm.clone(), "e_cur": e.clone(), "x_best": xm.clone(), "e_best": e.clone(),
                "stepsize": torch.full((W,), 0.4, dtype=torch.float64, device="cuda"),
                "win_accept": torch.zeros(W, dtype=torch.int32, device="cuda"),
                "n_accept": torch.zeros(W, dtype=torch.int32, device="cuda")}

    p = lj.BhParams(K=K, kT=0.8, seed=seed, n_steps=5, min=lj.LbfgsParams(prec=2))
    ref = fresh()
    lj.bh_step_batched(ctx, ref, p)
    lj.bh_step_batched(ctx, ref, p)       # same step0: the graph below replays it twice
    torch.cuda.synchronize()
    st = fresh()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        lj.bh_step_batched(ctx, st, p)
    init = fresh()
    for k in st:
        st[k].copy_(init[k])
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for k in st:
        assert torch.equal(st[k], ref[k]), k
    ctx.close()
