"""Writes the stored expected values under tests/golden/ from the FP64 oracle only.

lj38_oh_truncated_octahedron.txt: the LJ38 global minimum, which the paper's
Results describe as the compact truncated octahedron of O_h symmetry (the
discussion of the representative low-energy LJ38 structures).  The ideal fcc
truncated octahedron (nearest-neighbour distance 2^(1/6) sigma, eps = sigma =
1) is minimised by the oracle to ||grad E||_inf < 1e-6; its energy and
coordinates are written out.

Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
import oracle as O  # noqa: E402


def truncated_octahedron_38():
    pts = []
    for x in range(-3, 4):
        for y in range(-3, 4):
            for z in range(-3, 4):
                if (x + y + z) % 2 == 0:                 # fcc sites of the cubic lattice
                    d = np.array([x - 1.0, y, z])        # centred on the hole at (1, 0, 0)
                    if d @ d <= 5.0 + 1e-9:
                        pts.append(d)
    pts = np.array(pts)
    assert len(pts) == 38
    return pts * (2.0 ** (1.0 / 6.0) / math.sqrt(2.0))


def main():
    O.build()
    xm, em, st, _, _ = O.minimize(truncated_octahedron_38().reshape(-1))
    assert st == O.CONVERGED
    p = xm.reshape(38, 3)
    p = p - p.mean(0)
    path = os.path.join(HERE, "lj38_oh_truncated_octahedron.txt")
    with open(path, "w") as f:
        f.write("# LJ38 global minimum: truncated octahedron, O_h symmetry (paper, Results: the\n")
        f.write("# low-energy LJ38 structures). Written by tests/golden/make_golden.py from the FP64\n")
        f.write("# oracle (ideal fcc truncated octahedron minimised to ||grad E||_inf < 1e-6,\n")
        f.write("# eps = sigma = 1), centred on its centroid.\n")
        f.write(f"energy {em:.17g}\n")
        for r in p:
            f.write(f"{r[0]:.17g} {r[1]:.17g} {r[2]:.17g}\n")
    print(path, em)


if __name__ == "__main__":
    main()
