"""Seeded synthetic molecules and self-defined contracted Cartesian bases.

The paper validates on molecules and published basis sets that are not
available here, so every workload is synthetic (recipes below).  This module
only draws numbers: atom positions, nuclear charges, primitive exponents and
raw (unnormalised) contraction coefficients.  Normalisation, integrals and
everything else of the method live on each side separately (the CPU oracle and
the CUDA library).

Recipes
-------
* Element basis: for each angular momentum l a number of shells, each with 3
  primitives of even-tempered exponents a0 * 2.5**k (k = 0, 1, 2); a0 is drawn
  uniformly in [0.1, 0.5] per shell, shells of equal l on one element keep an
  a0 ratio >= 1.3 (rejection) so they are not near-duplicates; raw coefficients
  are uniform in (0.1, 1.0].  A basis is drawn once per element, in ascending Z.
* Water (small case): O at the origin, H at (+-1.4305, 1.1093, 0) bohr; O has
  3 s + 2 p shells, H 2 s shells; 10 electrons.
* Water cluster (H2O)_n: monomers of the small-case geometry, each rotated by a
  uniform random quaternion about O; O centres uniform in a cube of side
  12 * (n/8)**(1/3) bohr with O-O >= 5 bohr (rejection); O adds one d shell.
* Organic-like cloud: n heavy atoms on a jittered cubic lattice (spacing
  2.8 bohr, side ceil(n**(1/3)) sites, jitter U[-0.3, 0.3] per axis),
  Z in {6, 7, 8} with probabilities 0.70/0.15/0.15; heavy atoms carry
  4 s + 3 p + 1 d shells; when the electron count is odd one H (2 s + 1 p) is
  placed 2.0 bohr from a drawn heavy atom along a drawn direction, redrawn
  while closer than 1.8 bohr to any other atom.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64

# Offset that separates the geometry stream of a workload from its basis stream.
GEOM_STREAM = 1 << 40

WATER_O = (0.0, 0.0, 0.0)
WATER_H = ((1.4305, 1.1093, 0.0), (-1.4305, 1.1093, 0.0))


@dataclass(frozen=True)
class Shell:
    atom: int
    l: int
    alpha: tuple
    coef: tuple


@dataclass
class Molecule:
    name: str
    Z: list
    xyz: np.ndarray  # (natom, 3) bohr
    shells: list = field(default_factory=list)

    @property
    def natom(self) -> int:
        return len(self.Z)

    @property
    def nelec(self) -> int:
        return int(sum(self.Z))

    @property
    def nshell(self) -> int:
        return len(self.shells)

    @property
    def nbf(self) -> int:
        return sum((s.l + 1) * (s.l + 2) // 2 for s in self.shells)

    def arrays(self) -> dict:
        """Flat contiguous arrays (the layout the C interfaces take)."""
        nprim = np.array([len(s.alpha) for s in self.shells], dtype=np.int32)
        return {
            "Z": np.asarray(self.Z, dtype=np.int32),
            "xyz": np.ascontiguousarray(self.xyz, dtype=np.float64),
            "shell_atom": np.array([s.atom for s in self.shells], dtype=np.int32),
            "shell_l": np.array([s.l for s in self.shells], dtype=np.int32),
            "shell_nprim": nprim,
            "alpha": np.array([a for s in self.shells for a in s.alpha], dtype=np.float64),
            "coef": np.array([c for s in self.shells for c in s.coef], dtype=np.float64),
        }


def draw_element_basis(rng: SplitMix64, counts: dict, nprim: int = 3,
                       ratio: float = 2.5, min_sep: float = 1.3) -> list:
    """[(l, alphas, coefs), ...] for one element; counts maps l -> #shells."""
    out = []
    for l in sorted(counts):
        a0s: list = []
        tries = 0
        while len(a0s) < counts[l]:
            tries += 1
            if tries > 10000:  # restart a dead end
                a0s, tries = [], 0
            a0 = rng.uniform(0.1, 0.5)
            if all(max(a0, b) / min(a0, b) >= min_sep for b in a0s):
                a0s.append(a0)
        for a0 in a0s:
            alphas = tuple(a0 * ratio ** k for k in range(nprim))
            coefs = tuple(rng.uniform_open_low(0.1, 1.0) for _ in range(nprim))
            out.append((l, alphas, coefs))
    return out


def draw_basis_set(seed: int, element_counts: dict) -> dict:
    """Per-element bases drawn once from one stream in ascending Z."""
    rng = SplitMix64(seed)
    return {Z: draw_element_basis(rng, element_counts[Z]) for Z in sorted(element_counts)}


def _attach(name, Z, xyz, basis) -> Molecule:
    shells = []
    for ia, z in enumerate(Z):
        for (l, al, co) in basis[z]:
            shells.append(Shell(ia, l, al, co))
    return Molecule(name, list(Z), np.asarray(xyz, dtype=np.float64), shells)


def _quat_rotation(rng: SplitMix64) -> np.ndarray:
    """Uniform random rotation (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    w, x, y, z = (a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                  b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3))
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


WATER_BASIS_COUNTS = {1: {0: 2}, 8: {0: 3, 1: 2}}
CLUSTER_BASIS_COUNTS = {1: {0: 2}, 8: {0: 3, 1: 2, 2: 1}}
ORGANIC_BASIS_COUNTS = {1: {0: 2, 1: 1}, 6: {0: 4, 1: 3, 2: 1},
                        7: {0: 4, 1: 3, 2: 1}, 8: {0: 4, 1: 3, 2: 1}}


def water(seed: int = 0) -> Molecule:
    """One water molecule, O 3s2p / H 2s, basis drawn from `seed`."""
    basis = draw_basis_set(seed, WATER_BASIS_COUNTS)
    return _attach("water", [8, 1, 1], [WATER_O, *WATER_H], basis)


def water_cluster(nmono: int = 8, geom_seed: int = 1, basis_seed: int = 1,
                  min_oo: float = 5.0) -> Molecule:
    """(H2O)_n with rotated monomers in a cube scaled to keep 8 per 12^3 bohr^3."""
    basis = draw_basis_set(basis_seed, CLUSTER_BASIS_COUNTS)
    rng = SplitMix64(geom_seed + GEOM_STREAM)
    side = 12.0 * (nmono / 8.0) ** (1.0 / 3.0)
    centres: list = []
    while len(centres) < nmono:
        c = np.array([rng.uniform(0.0, side) for _ in range(3)])
        if all(np.linalg.norm(c - o) >= min_oo for o in centres):
            centres.append(c)
    Z, xyz = [], []
    for c in centres:
        R = _quat_rotation(rng)
        Z += [8, 1, 1]
        xyz.append(c)
        for h in WATER_H:
            xyz.append(c + R @ np.array(h))
    return _attach(f"(H2O)_{nmono}", Z, xyz, basis)


def organic_cloud(nheavy: int = 60, geom_seed: int = 2, basis_seed: int = 2,
                  spacing: float = 2.8, jitter: float = 0.3) -> Molecule:
    """Heavy-atom cloud on a jittered lattice, H-capped to an even electron count."""
    basis = draw_basis_set(basis_seed, ORGANIC_BASIS_COUNTS)
    rng = SplitMix64(geom_seed + GEOM_STREAM)
    k = 1
    while k ** 3 < nheavy:
        k += 1
    sites = [(i, j, m) for i in range(k) for j in range(k) for m in range(k)]
    rng.shuffle(sites)
    Z, xyz = [], []
    for s in sites[:nheavy]:
        xyz.append(np.array([spacing * s[d] + rng.uniform(-jitter, jitter) for d in range(3)]))
        Z.append((6, 7, 8)[rng.choice((0.70, 0.15, 0.15))])
    if sum(Z) % 2 == 1:
        while True:
            a = rng.randint(0, nheavy - 1)
            v = np.array([rng.normal() for _ in range(3)])
            v /= np.linalg.norm(v)
            h = xyz[a] + 2.0 * v
            if all(np.linalg.norm(h - x) >= 1.8 for x in xyz):
                break
        Z.append(1)
        xyz.append(h)
    return _attach(f"cloud_{nheavy}", Z, np.array(xyz), basis)


def batched_set(nmol: int = 512, seed: int = 3, nmin: int = 3, nmax: int = 30,
                basis_seed: int = 2) -> list:
    """Uneven batch: heavy-atom counts uniform on [nmin, nmax], clouds as above."""
    rng = SplitMix64(seed)
    sizes = [rng.randint(nmin, nmax) for _ in range(nmol)]
    return [organic_cloud(n, geom_seed=(seed << 32) + i, basis_seed=basis_seed)
            for i, n in enumerate(sizes)]


def workload(name: str) -> Molecule:
    """Named single-molecule workloads."""
    if name == "water":
        return water(0)
    if name == "water8":
        return water_cluster(8, geom_seed=1, basis_seed=1)
    if name == "cloud60":
        return organic_cloud(60, geom_seed=2, basis_seed=2)
    if name.startswith("cloud"):
        return organic_cloud(int(name[5:]), geom_seed=2, basis_seed=2)
    if name.startswith("water") and name[5:].isdigit():
        return water_cluster(int(name[5:]), geom_seed=1, basis_seed=1)
    raise KeyError(name)
