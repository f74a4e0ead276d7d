"""Molden input/output (host side): the first geometry of a file becomes the
flattened 3N coordinate vector, accepted structures are appended as XYZ
frames, and what is written reads back unchanged."""
import numpy as np
import pytest

from paper_2510_25938_gb300 import molden


def test_write_then_read_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    frames = [molden.Geometry(["Ar"] * 5, rng.normal(size=(5, 3)) * 2.0, f"step {i} energy -9.1")
              for i in range(3)]
    path = str(tmp_path / "x_accepted.molden")
    molden.write_geometries(path, frames[:1], append=False)
    molden.write_geometries(path, frames[1:])          # append: frames only
    text = open(path).read()
    assert text.startswith("[Molden Format]\n[GEOMETRIES] XYZ\n")
    assert text.count("[GEOMETRIES]") == 1
    back = molden.read_geometries(path)
    assert len(back) == 3
    for a, b in zip(frames, back):
        assert b.symbols == a.symbols and b.comment == a.comment
        assert np.allclose(b.coords, a.coords, atol=1e-11, rtol=0)
    first = molden.read_first_geometry(path)
    assert np.allclose(first.flat, frames[0].coords.reshape(-1), atol=1e-11, rtol=0)


def test_atoms_section_in_angstrom_and_atomic_units(tmp_path):
    body = ("[Molden Format]\n[Title]\ncluster\n[Atoms] {unit}\n"
            "Ar 1 18 0.0 0.0 0.0\nAr 2 18 1.5 0.0 0.0\nAr 3 18 0.0 2.0 -1.0\n"
            "[GTO]\n")
    p1 = tmp_path / "a.molden"
    p1.write_text(body.format(unit="Angs"))
    g = molden.read_first_geometry(str(p1))
    assert g.symbols == ["Ar"] * 3
    assert g.flat.tolist() == [0, 0, 0, 1.5, 0, 0, 0, 2, -1]
    p2 = tmp_path / "b.molden"
    p2.write_text(body.format(unit="AU"))
    g2 = molden.read_first_geometry(str(p2))
    assert np.allclose(g2.flat, g.flat * molden.BOHR_IN_ANGSTROM, rtol=1e-15, atol=0)


def test_bare_xyz_and_first_of_several_frames(tmp_path):
    p = tmp_path / "c.xyz"
    p.write_text("2\nfirst\nX 0 0 0\nX 1.1 0 0\n2\nsecond\nX 0 0 0\nX 9 0 0\n")
    g = molden.read_first_geometry(str(p))
    assert g.comment == "first" and g.flat.tolist() == [0, 0, 0, 1.1, 0, 0]


def test_accepted_path_and_bad_input(tmp_path):
    assert molden.accepted_path("/a/b/lj38.molden") == "/a/b/lj38_accepted.molden"
    p = tmp_path / "bad.molden"
    p.write_text("[Molden Format]\n[Title]\nnothing here\n")
    with pytest.raises(ValueError):
        molden.read_first_geometry(str(p))
