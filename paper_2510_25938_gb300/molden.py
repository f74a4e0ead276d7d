"""Molden geometry files: the input and output format of the method's driver.

The paper's program reads the first geometry of a ``.molden`` file and
flattens it into the 3N coordinate vector the minimiser works on
(Methodology, "Initial Structures and Input"), and appends every accepted
structure to ``<input>_accepted.molden`` ("Running the Code").  This module
does both on the host; it holds no part of the method's arithmetic.

Reading understands the two common layouts of a Molden file:

* an ``[Atoms]`` section (``[Atoms] Angs`` or ``[Atoms] AU``), one atom per
  line as ``name number atomic_number x y z``;
* a ``[GEOMETRIES] XYZ`` section followed by XYZ frames (atom count, comment
  line, ``symbol x y z`` lines) -- the first frame is taken;

and a bare XYZ file.  Coordinates in atomic units are converted to
Angstrom.  Lennard-Jones runs use reduced units (eps = sigma = 1), so the
numbers are then taken as lengths in units of sigma.

Writing produces a ``[Molden Format]`` file with a ``[GEOMETRIES] XYZ``
section, one XYZ frame per structure; appending to an existing file adds
frames only.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

BOHR_IN_ANGSTROM = 0.529177210903


@dataclass
class Geometry:
    symbols: list
    coords: np.ndarray          # (N, 3) float64
    comment: str = ""

    @property
    def flat(self) -> np.ndarray:
        """The flattened 3N coordinate vector (x1, y1, z1, x2, ...)."""
        return np.ascontiguousarray(self.coords, dtype=np.float64).reshape(-1)


def _section(line: str) -> str | None:
    s = line.strip()
    if s.startswith("[") and "]" in s:
        return s[1:s.index("]")].strip().lower()
    return None


def _parse_xyz_frame(lines, i):
    """XYZ frame starting at lines[i] (the atom count); returns (Geometry, next index)."""
    n = int(lines[i].split()[0])
    comment = lines[i + 1].rstrip("\n") if i + 1 < len(lines) else ""
    symbols, xyz = [], []
    for k in range(n):
        parts = lines[i + 2 + k].split()
        symbols.append(parts[0])
        xyz.append([float(v) for v in parts[1:4]])
    return Geometry(symbols, np.array(xyz, dtype=np.float64).reshape(n, 3), comment), i + 2 + n


def read_first_geometry(path: str) -> Geometry:
    """The first geometry of a Molden (or XYZ) file."""
    with open(path) as f:
        lines = f.readlines()
    i = 0
    while i < len(lines):
        sec = _section(lines[i])
        if sec is not None and sec.startswith("atoms"):
            unit = lines[i].strip()[lines[i].index("]") + 1:].strip().lower()
            scale = BOHR_IN_ANGSTROM if unit.startswith("au") or unit.startswith("bohr") else 1.0
            symbols, xyz = [], []
            i += 1
            while i < len(lines) and lines[i].strip() and _section(lines[i]) is None:
                parts = lines[i].split()
                symbols.append(parts[0])
                xyz.append([float(v) * scale for v in parts[3:6]])
                i += 1
            if not symbols:
                raise ValueError(f"{path}: empty [Atoms] section")
            return Geometry(symbols, np.array(xyz, dtype=np.float64))
        if sec is not None and sec.startswith("geometries"):
            i += 1
            while i < len(lines) and not lines[i].strip():
                i += 1
            return _parse_xyz_frame(lines, i)[0]
        i += 1
    # a bare XYZ file
    i = 0
    while i < len(lines) and not lines[i].strip():
        i += 1
    if i < len(lines) and lines[i].split() and lines[i].split()[0].isdigit():
        return _parse_xyz_frame(lines, i)[0]
    raise ValueError(f"{path}: no [Atoms] or [GEOMETRIES] section and not an XYZ file")


def read_geometries(path: str) -> list:
    """Every XYZ frame of a file written by write_geometries (or any file
    whose [GEOMETRIES] XYZ section holds consecutive frames)."""
    with open(path) as f:
        lines = f.readlines()
    frames, i = [], 0
    while i < len(lines) and not (_section(lines[i]) or "").startswith("geometries"):
        i += 1
    i += 1
    while i < len(lines):
        if not lines[i].strip():
            i += 1
            continue
        if _section(lines[i]) is not None:
            break
        g, i = _parse_xyz_frame(lines, i)
        frames.append(g)
    return frames


def _frame_text(g: Geometry) -> str:
    out = [f"{len(g.symbols)}\n", g.comment.replace("\n", " ") + "\n"]
    for s, (x, y, z) in zip(g.symbols, np.asarray(g.coords).reshape(-1, 3)):
        out.append(f"{s:<3s} {x: .12f} {y: .12f} {z: .12f}\n")
    return "".join(out)


def write_geometries(path: str, frames, append: bool = True) -> None:
    """Write (or append) XYZ frames under a [GEOMETRIES] XYZ section."""
    new = not append or not os.path.exists(path) or os.path.getsize(path) == 0
    with open(path, "w" if new else "a") as f:
        if new:
            f.write("[Molden Format]\n[GEOMETRIES] XYZ\n")
        for g in frames:
            f.write(_frame_text(g))


def accepted_path(input_path: str) -> str:
    """<input>_accepted.molden next to the input file."""
    root, _ = os.path.splitext(input_path)
    return root + "_accepted.molden"
