"""lbfgs_minimize_batched_noalloc against lbfgs_minimize_batched.

The no-allocation entry point is for callers that must not allocate device
memory (a CUDA graph being captured, an application whose memory manager owns
the device memory, latency-critical loops): it keeps its scratch in a fixed
library array instead of a context workspace.  It must give the results of
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
