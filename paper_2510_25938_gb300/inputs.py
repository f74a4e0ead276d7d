"""Seeded synthetic inputs for batched LJ minimisation and Basin Hopping.

This module only makes starting coordinates; it holds none of the method's
arithmetic (no energies, no minimisation, no Basin Hopping step).  Both the
CUDA path and the CPU oracle are fed from it.  Random numbers come from numpy's
PCG64 seeded per workload; the random numbers the method itself draws
(perturbations, Metropolis uniforms) come from the Philox streams that each
side implements on its own.

Workload shapes (arXiv 2510.25938 uses LJ clusters, LJ38 as the hard case,
200 BH steps and up to eight concurrent candidates; the batch sizes are this
library's):

* cube starts: N atoms uniform in [0, L)^3 (L = 2.0 sigma for N=13,
  3.2 sigma for N=38, or L = (N / rho)^(1/3) for a reduced density rho);
* uneven batches: N ~ U{lo..hi} per candidate, cube at density 0.3;
* fcc fragments: the N fcc sites nearest the origin (nearest-neighbour
  distance 2^(1/6) sigma), then Gaussian jitter;
* jittered configurations: Gaussian jitter of given coordinates.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 2510259380


def workload_seed(config_id: int) -> int:
    return SEED_BASE + int(config_id)


def cube_side_for_density(n_atoms: int, rho: float) -> float:
    return float((n_atoms / rho) ** (1.0 / 3.0))


def cube_starts(n_cand: int, n_atoms: int, side: float, seed: int) -> np.ndarray:
    """(n_cand, 3N) float64, every coordinate uniform in [0, side)."""
    rng = np.random.default_rng(seed)
    return rng.random((n_cand, 3 * n_atoms)) * side


def uneven_sizes(n_cand: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Atom counts uniform on {lo..hi} (inclusive)."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=n_cand).astype(np.int64)


def offsets_from_sizes(sizes) -> np.ndarray:
    sizes = np.asarray(sizes, dtype=np.int64)
    off = np.zeros(sizes.size + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def uneven_cube_starts(sizes, rho: float, seed: int):
    """Packed coordinates (total_atoms*3,) and offsets (n_cand+1,) for clusters
    of the given sizes, each uniform in a cube of reduced density rho."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    off = offsets_from_sizes(sizes)
    x = np.empty(3 * int(off[-1]))
    for c, n in enumerate(sizes):
        side = cube_side_for_density(int(n), rho)
        x[3 * off[c]:3 * off[c + 1]] = rng.random(3 * int(n)) * side
    return x, off


def fcc_sites(n_atoms: int, nn_dist: float = 2.0 ** (1.0 / 6.0)) -> np.ndarray:
    """The n_atoms fcc lattice sites closest to a lattice site at the origin,
    ties broken by (r^2, x, y, z); (n_atoms, 3)."""
    a = nn_dist * np.sqrt(2.0)                     # cubic lattice constant
    k = int(np.ceil((n_atoms / 4.0) ** (1.0 / 3.0))) + 2
    rng_ = np.arange(-k, k + 1)
    cx, cy, cz = np.meshgrid(rng_, rng_, rng_, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1).astype(np.float64)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    pts = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    r2 = np.round((pts ** 2).sum(1), 9)
    order = np.lexsort((np.round(pts[:, 2], 9), np.round(pts[:, 1], 9),
                        np.round(pts[:, 0], 9), r2))
    return pts[order[:n_atoms]].copy()


def jitter(x: np.ndarray, sigma_x: float, seed: int) -> np.ndarray:
    """x + N(0, sigma_x^2) per coordinate (x any shape)."""
    rng = np.random.default_rng(seed)
    return x + rng.normal(0.0, sigma_x, size=x.shape)


def fcc_fragments(n_cand: int, n_atoms: int, sigma_x: float, seed: int) -> np.ndarray:
    """(n_cand, 3N): the fcc fragment with independent Gaussian jitter."""
    base = fcc_sites(n_atoms).reshape(1, -1)
    return jitter(np.repeat(base, n_cand, axis=0), sigma_x, seed)
