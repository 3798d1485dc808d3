"""Small hand-made molecules for pins (raw shells; normalisation is per side)."""
import numpy as np

from fsim_synth import Molecule, Shell


def make_mol(atoms, shells, name="test"):
    """atoms: [(Z, (x, y, z)), ...]; shells: [(atom, l, alphas, coefs), ...]."""
    Z = [a[0] for a in atoms]
    xyz = np.array([a[1] for a in atoms], dtype=float)
    sh = [Shell(s[0], s[1], tuple(s[2]), tuple(s[3])) for s in shells]
    return Molecule(name, Z, xyz, sh)


def random_mol(rng, natom=3, lmax=2, nprim=1, spread=2.0, name="rand"):
    """Random small molecule: one shell of each l <= lmax per atom."""
    atoms, shells = [], []
    for a in range(natom):
        atoms.append((int(rng.integers(1, 9)), tuple(rng.uniform(-spread, spread, 3))))
        for l in range(lmax + 1):
            al = tuple(sorted(rng.uniform(0.2, 2.5, nprim)))
            co = tuple(rng.uniform(0.2, 1.0, nprim))
            shells.append((a, l, al, co))
    return make_mol(atoms, shells, name)
