"""lbfgs_minimize_batched_noalloc against lbfgs_minimize_batched.

The no-allocation entry point is for callers that must not allocate device
memory (an application whose memory manager owns the device memory, code
where an allocation's device synchronisation is not acceptable,
latency-critical loops): it keeps its scratch in a fixed library array
instead of a context workspace.  It must give the results of
the ordinary entry point, on two calls in a row (the scratch array is shared
between calls and keeps the previous call's contents).  This file is named to
run last, and passes on its own as well as after the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2510_25938_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_REL_E = 1e-10
MIX_ABS_FINAL = 1e-6


@pytest.fixture(scope="module")
def lj():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25938_gb300 import build
    build.build()
    from paper_2510_25938_gb300 import lj_bh
    torch.cuda.set_device(0)
    return lj_bh


def _run_ctx(lj, x0, off, prec):
    ctx = lj.Ctx(0)
    n_cand = off.size - 1
    x = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
    e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
    st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
    lj.lbfgs_minimize_batched(ctx, x, e, st, n_cand=n_cand,
                              atom_offset=torch.as_tensor(off, device="cuda"),
                              max_n=int(np.diff(off).max()), params=lj.LbfgsParams(prec=prec))
    torch.cuda.synchronize()
    ctx.close()
    return x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()


def _run_noalloc_c(lj, x0, off, prec):
    """Straight through the C entry point (ctypes), no context."""
    lib = lj.load()
    n_cand = off.size - 1
    x = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
    e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
    st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
    it = torch.empty(n_cand, dtype=torch.int32, device="cuda")
    stats = lj.new_stats()
    offd = torch.as_tensor(off, device="cuda")
    b = lj._Batch(n_cand, 0, offd.data_ptr(), int(np.diff(off).max()))
    p = lj.LbfgsParams(prec=prec).c()
    rc = lib.lbfgs_minimize_batched_noalloc(C.byref(b), C.byref(p), x.data_ptr(), e.data_ptr(),
                                            st.data_ptr(), it.data_ptr(), None,
                                            stats.data_ptr(),
                                            torch.cuda.current_stream().cuda_stream)
    assert rc == lj.LJ_OK
    torch.cuda.synchronize()
    return x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy(), lj.stats_dict(stats)


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("case", ["lj38", "uneven"])
def test_noalloc_matches_context_entry_point_on_two_calls(lj, prec, case):
    if case == "lj38":
        n_cand = 96
        x0 = I.cube_starts(n_cand, 38, 3.2, I.workload_seed(1) + 50).reshape(-1)
        off = np.arange(n_cand + 1, dtype=np.int64) * 38
    else:
        sizes = I.uneven_sizes(40, 13, 150, I.workload_seed(3))
        x0, off = I.uneven_cube_starts(sizes, 0.3, I.workload_seed(3) + 1)
    xr, er, sr = _run_ctx(lj, x0, off, prec)
    first = None
    for call in range(2):
        xg, eg, sg, stats = _run_noalloc_c(lj, x0, off, prec)
        assert stats["minimisations"] == off.size - 1
        assert np.array_equal(sg, sr)
        fin = np.isfinite(er)
        if prec == 0:
            assert np.all(np.abs(eg[fin] - er[fin]) <= FP64_REL_E * np.abs(er[fin]))
        else:
            assert np.all(np.abs(eg[fin] - er[fin]) <= MIX_ABS_FINAL)
        if first is None:
            first = (xg, eg)
        else:                            # the second call repeats the first
            assert np.array_equal(first[0], xg) and np.array_equal(first[1], eg)


def test_noalloc_large_clusters_with_capped_grid(lj):
    """600-atom FP64 minimisations with m = 20: each team's history (2 m x 3 x
    1024 doubles, ~983 KB) lives off chip, only ~17 slots fit in the scratch
    array, so the launch is capped below the batch size and teams take several
    candidates each from the queue.  Results equal the context entry point's,
    twice in a row."""
    n_cand, n_atoms = 20, 600
    x0 = I.fcc_fragments(n_cand, n_atoms, 0.1, I.workload_seed(4) + 600).reshape(-1)
    off = np.arange(n_cand + 1, dtype=np.int64) * n_atoms

    def run(noalloc):
        x = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
        e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
        st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
        stats = lj.new_stats()
        p = lj.LbfgsParams(prec=lj.LJ_PREC_FP64, m=20)
        if noalloc:
            lib = lj.load()
            b = lj._Batch(n_cand, n_atoms, None, n_atoms)
            pc = p.c()
            rc = lib.lbfgs_minimize_batched_noalloc(C.byref(b), C.byref(pc), x.data_ptr(),
                                                    e.data_ptr(), st.data_ptr(), None, None,
                                                    stats.data_ptr(),
                                                    torch.cuda.current_stream().cuda_stream)
            assert rc == lj.LJ_OK
        else:
            ctx = lj.Ctx(0)
            lj.lbfgs_minimize_batched(ctx, x, e, st, None, None, stats, n_cand=n_cand,
                                      uniform_n=n_atoms, params=p)
            torch.cuda.synchronize()
            ctx.close()
        torch.cuda.synchronize()
        return x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy(), lj.stats_dict(stats)

    xr, er, sr, _ = run(False)
    assert np.all(sr == 0)
    for call in range(2):
        xg, eg, sg, stats = run(True)
        assert stats["minimisations"] == n_cand
        assert np.array_equal(sg, sr)
        assert np.all(np.abs(eg - er) <= FP64_REL_E * np.abs(er))


@pytest.mark.parametrize("prec", [0, 2])
def test_noalloc_morse_matches_context_entry_point(lj, prec):
    """The no-allocation entry point takes the pair potential from the same
    parameters (Morse, rho = 6, an uneven batch across buckets): results equal
    the context entry point's."""
    sizes = I.uneven_sizes(24, 8, 80, I.workload_seed(3) + 70)
    x0, off = I.uneven_cube_starts(sizes, 0.3, I.workload_seed(3) + 71)
    n_cand = off.size - 1
    p = lj.LbfgsParams(prec=prec, potential=lj.LJ_POT_MORSE, rho=6.0)
    offd = torch.as_tensor(off, device="cuda")

    def run(noalloc):
        x = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
        e = torch.empty(n_cand, dtype=torch.float64, device="cuda")
        st = torch.empty(n_cand, dtype=torch.int32, device="cuda")
        if noalloc:
            lib = lj.load()
            b = lj._Batch(n_cand, 0, offd.data_ptr(), int(np.diff(off).max()))
            pc = p.c()
            rc = lib.lbfgs_minimize_batched_noalloc(C.byref(b), C.byref(pc), x.data_ptr(),
                                                    e.data_ptr(), st.data_ptr(), None, None, None,
                                                    torch.cuda.current_stream().cuda_stream)
            assert rc == lj.LJ_OK
        else:
            ctx = lj.Ctx(0)
            lj.lbfgs_minimize_batched(ctx, x, e, st, n_cand=n_cand, atom_offset=offd,
                                      max_n=int(np.diff(off).max()), params=p)
            torch.cuda.synchronize()
            ctx.close()
        torch.cuda.synchronize()
        return x.cpu().numpy(), e.cpu().numpy(), st.cpu().numpy()

    xr, er, sr = run(False)
    xg, eg, sg = run(True)
    assert np.array_equal(sg, sr)
    fin = np.isfinite(er)
    tol = FP64_REL_E * np.abs(er[fin]) if prec == 0 else MIX_ABS_FINAL
    assert np.all(np.abs(eg[fin] - er[fin]) <= tol)
