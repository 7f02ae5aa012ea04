"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers and lays them out as arrays.  It holds
none of the method's arithmetic (no grid placement, no discretisation, no
energies), so the oracle and the GPU library can both take their inputs from it
without sharing any part of the computation.

Atoms are rows ``(x, y, z, R, q)`` in Angstrom and elementary charges, float64,
C-contiguous, shape ``(N, 5)``.

Workload shapes (the paper's biomolecular systems are not available here, so
these synthetic molecules stand in for them):

* globular molecule: centres uniform in a ball of radius ``R_b`` by random
  sequential addition with a 1.5 A minimum spacing, radii U[1.2, 2.0] A,
  charges N(0, 0.4) e rounded to 0.01 e, no neutralisation;
  ``R_b = 20 * (N / 2000) ** (1/3)`` A unless given.
* Born ion: one +1 e charge of radius 2 A at (10, 10, 10) in a 20 A box.
* batch: molecule ``i`` of a batch uses seed ``seed_base + i`` and an atom
  count log-uniform in ``[lo, hi]`` drawn from ``seed_base``.
"""
from __future__ import annotations

import math

import numpy as np

MIN_SPACING = 1.5
RADIUS_RANGE = (1.2, 2.0)
CHARGE_SIGMA = 0.4


def ball_radius(n_atoms: int) -> float:
    """Radius of the ball holding ``n_atoms`` centres at the 2000-atom density."""
    return 20.0 * (n_atoms / 2000.0) ** (1.0 / 3.0)


def globular_molecule(n_atoms: int, seed: int, radius: float | None = None,
                      center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Random-sequential-addition molecule; see the module docstring."""
    if n_atoms < 1:
        raise ValueError("n_atoms must be >= 1")
    rb = ball_radius(n_atoms) if radius is None else float(radius)
    rng = np.random.Generator(np.random.PCG64(seed))
    cell = MIN_SPACING
    occupied: dict[tuple[int, int, int], list[int]] = {}
    pts = np.empty((n_atoms, 3))
    count = 0
    attempts = 0
    max_attempts = 200 * n_atoms + 10000
    d2min = MIN_SPACING * MIN_SPACING
    while count < n_atoms:
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError("random sequential addition did not converge")
        # uniform in the ball: direction from a normal draw, radius ~ u^(1/3)
        v = rng.normal(size=3)
        nv = math.sqrt(float(v @ v))
        if nv == 0.0:
            continue
        r = rb * rng.random() ** (1.0 / 3.0)
        p = v * (r / nv)
        key = (int(math.floor(p[0] / cell)), int(math.floor(p[1] / cell)),
               int(math.floor(p[2] / cell)))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in occupied.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        d = pts[j] - p
                        if float(d @ d) < d2min:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if not ok:
            continue
        pts[count] = p
        occupied.setdefault(key, []).append(count)
        count += 1
    radii = rng.uniform(RADIUS_RANGE[0], RADIUS_RANGE[1], size=n_atoms)
    charges = np.round(rng.normal(0.0, CHARGE_SIGMA, size=n_atoms), 2)
    atoms = np.empty((n_atoms, 5))
    atoms[:, :3] = pts + np.asarray(center, dtype=np.float64)
    atoms[:, 3] = radii
    atoms[:, 4] = charges
    return np.ascontiguousarray(atoms)


def born_ion() -> np.ndarray:
    """One +1 e charge at the centre of a 2 A sphere, placed at (10, 10, 10)."""
    return np.array([[10.0, 10.0, 10.0, 2.0, 1.0]])


def lattice_balls() -> np.ndarray:
    """Balls placed on the lattice of spacing 0.5 from (-8, -8, -8): surfaces
    through nodes (interval ends exactly at 0 or 1), spheres tangent to
    lattice lines, a chord inside one edge, nested and abutting balls, and
    two partial intervals whose union is a whole edge."""
    return np.array([
        [0.0, 0.0, 0.0, 2.0, 1.0],      # centre on a node, R = 4h
        [0.0, 0.0, 0.0, 1.0, 0.0],      # nested, same centre
        [3.0, 0.0, 0.0, 1.0, -1.0],     # touches the first at the node x = 2
        [-4.0, 2.75, 1.0, 0.25, 0.5],   # tangent to the lines y = 2.5 and 3.0 at z = 1
        [5.25, 5.0, 5.0, 0.2, 0.0],     # chord [5.05, 5.45] inside the edge [5, 5.5]
        [-5.0, -5.0, 4.0, 0.65, 0.3],   # covers [-5.5, -5.0] and part of [-4.5, -4.0] ...
        [-4.0, -5.0, 4.0, 0.55, 0.0],   # ... and this one the rest of it
        [4.0, -4.0, -4.0, 1.5, -0.5],   # centre on a node, R = 3h
        [4.25, -4.25, -3.75, 0.75, 0.0],  # centre at a cell centre
    ])


def snapped_molecule(n_atoms: int = 80, seed: int = 104) -> np.ndarray:
    """A globular molecule centred on the origin with coordinates rounded to
    multiples of 0.125 and radii to multiples of 0.25 (at least 0.5): on the
    lattice of spacing 0.5 its spheres meet nodes and lines exactly."""
    atoms = globular_molecule(n_atoms, seed=seed)
    atoms[:, :3] = np.round((atoms[:, :3] - atoms[:, :3].mean(0)) / 0.125) * 0.125
    atoms[:, 3] = np.maximum(np.round(atoms[:, 3] / 0.25) * 0.25, 0.5)
    return atoms


def batch_sizes(count: int, seed_base: int, lo: int, hi: int) -> np.ndarray:
    """Atom counts log-uniform in [lo, hi] for a batch of ``count`` molecules."""
    rng = np.random.Generator(np.random.PCG64(seed_base))
    u = rng.random(count)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))).astype(np.int64).clip(lo, hi)


def batch_molecules(count: int, seed_base: int, lo: int = 200, hi: int = 3000) -> list[np.ndarray]:
    """``count`` globular molecules, molecule ``i`` seeded with ``seed_base + i``."""
    sizes = batch_sizes(count, seed_base, lo, hi)
    return [globular_molecule(int(n), seed_base + i) for i, n in enumerate(sizes)]


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard-normal test vector (used for operator-apply parity)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=shape).astype(dtype)


def poisson_arrivals(count: int, rate_hz: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with rate ``rate_hz``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
