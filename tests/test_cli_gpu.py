"""The command-line driver on the GPU (python -m paper_2510_25938_gb300
input.molden): the first geometry of the input is minimised and Basin
Hopping runs; the accepted-structure file opens with the minimised start,
then holds one frame per accepted step, each a local minimum whose FP64
energy (recomputed here) is the one written beside it."""
import json
import re

import numpy as np
import pytest

import oracle as O
from paper_2510_25938_gb300 import inputs as I
from paper_2510_25938_gb300 import molden
from tests.helpers import numpy_energy_grad, record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cli():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_25938_gb300 import build
    build.build()
    from paper_2510_25938_gb300 import cli as C
    return C


@pytest.mark.parametrize("precision,walkers", [("fp64", 1), ("mixed", 2)])
def test_cli_writes_accepted_minima(cli, tmp_path, capsys, precision, walkers):
    x0 = I.cube_starts(1, 13, 2.0, I.workload_seed(0) + 77).reshape(13, 3)
    src = tmp_path / "lj13.molden"
    molden.write_geometries(str(src), [molden.Geometry(["Ar"] * 13, x0, "cube start")],
                            append=False)
    rc = cli.main([str(src), "--steps", "30", "--candidates", "4", "--precision", precision,
                   "--walkers", str(walkers), "--json"])
    assert rc == 0
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert out["walkers"] == walkers and len(out["accepted_files"]) == walkers
    for w, path in enumerate(out["accepted_files"]):
        frames = molden.read_geometries(path)
        n_acc = round(out["acceptance_rate"][w] * 30)
        assert len(frames) == 1 + n_acc
        energies = []
        for g in frames:
            e_file = float(re.search(r"energy (\S+)", g.comment).group(1))
            e, grad = numpy_energy_grad(g.flat)
            assert abs(e - e_file) <= 1e-8 * abs(e)
            # a local minimum: converged ones to gtol (the coordinates are written
            # with 12 decimals), the rest (the selection keeps them eligible) close
            converged = "status" not in g.comment or "status converged" in g.comment
            assert np.abs(grad).max() < (1.01e-6 if converged else 1e-3)
            energies.append(e)
        assert min(energies) == pytest.approx(out["best_energy"][w], abs=1e-8)
        assert energies[-1] == pytest.approx(out["final_energy"][w], abs=1e-8)
        # the start frame is the oracle's minimum of the same start (FP64, LJ13)
        if precision == "fp64":
            _, eo, _, _, _ = O.lbfgs_batch(x0.reshape(-1), 1, uniform_n=13)
            assert abs(energies[0] - eo[0]) <= 1e-9 * abs(eo[0])
        record(f"cli_{precision}_w{w}", frames=len(frames), best=min(energies))
