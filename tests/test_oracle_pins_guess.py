"""Pins of the oracle's learned-guess geometry (oracle/guess.py).

The paper has no learned guess, so nothing prints values to compare with;
what fixes these functions is how they must behave under rotations:
hand-worked shell transforms (p: U = R; d: a quarter turn about z maps xx to
yy and flips xy), features invariant under a rigid motion of the molecule,
local blocks of a rotation-covariant matrix (the inverse overlap S^{-1}
transforms exactly like a density, D' = U^{-T} D U^{-1}) unchanged by the
rotation, and assembly undoing the local transform.
"""
import math

import numpy as np
import pytest

from fsim_synth import water_cluster
from oracle import OracleBasis
from oracle import guess as og

from .helpers import make_mol


def _rot(a, b, c):
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])
    Rx = np.array([[1.0, 0, 0], [0, math.cos(b), -math.sin(b)], [0, math.sin(b), math.cos(b)]])
    Ry = np.array([[math.cos(c), 0, math.sin(c)], [0, 1.0, 0], [-math.sin(c), 0, math.cos(c)]])
    return Rz @ Rx @ Ry


def _moved(mol, Q, t):
    return make_mol([(z, tuple(Q @ x + t)) for z, x in zip(mol.Z, mol.xyz)],
                    [(s.atom, s.l, s.alpha, s.coef) for s in mol.shells])


def test_shell_transforms_hand_worked():
    R = _rot(0.7, -0.4, 1.1)
    assert np.allclose(og.shell_U(0, R), [[1.0]], atol=1e-12)
    assert np.allclose(og.shell_U(1, R), R, atol=1e-12)
    # quarter turn about z: (x, y, z) -> (-y, x, z)
    Q = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    U = og.shell_U(2, Q)  # d components xx xy xz yy yz zz
    ref = np.zeros((6, 6))
    ref[0, 3] = 1.0   # (1/sqrt3) (-y)^2 = g_yy
    ref[1, 1] = -1.0  # (-y) x = -g_xy
    ref[2, 4] = -1.0  # (-y) z = -g_yz
    ref[3, 0] = 1.0   # x^2 / sqrt3 = g_xx
    ref[4, 2] = 1.0   # x z = g_xz
    ref[5, 5] = 1.0
    assert np.allclose(U, ref, atol=1e-12)
    # composition: g(R1 R2 v) = U(R1) g(R2 v) = U(R1) U(R2) g(v)
    R2 = _rot(-0.3, 0.9, 0.2)
    assert np.allclose(og.shell_U(2, R @ R2), og.shell_U(2, R) @ og.shell_U(2, R2), atol=1e-10)


def test_frames_are_rotations():
    mol = water_cluster(2, geom_seed=4)
    for A, B, R, f in og.pairs(mol):
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and np.linalg.det(R) == pytest.approx(1.0)
        if A != B:
            d = np.asarray(mol.xyz[B]) - np.asarray(mol.xyz[A])
            assert np.allclose(R[2], d / np.linalg.norm(d))
            assert f[0] == pytest.approx(0.1 * np.linalg.norm(d)) and f[47] == 0.0
        else:
            assert f[47] == 1.0 and f[0] == 0.0


def test_features_invariant_under_rigid_motion():
    mol = water_cluster(3, geom_seed=5)
    Q = _rot(1.3, 0.4, -2.0)
    moved = _moved(mol, Q, np.array([3.0, -1.0, 0.5]))
    assert np.abs(og.features(mol) - og.features(moved)).max() < 1e-12


@pytest.fixture(scope="module")
def dimer_pair():
    mol = water_cluster(2, geom_seed=6)
    moved = _moved(mol, _rot(-0.8, 2.1, 0.6), np.array([-1.0, 2.0, 0.3]))
    return mol, moved


def test_local_blocks_of_a_covariant_matrix_are_rotation_invariant(dimer_pair):
    mol, moved = dimer_pair
    D1 = np.linalg.inv(OracleBasis(mol).onee("S"))
    D2 = np.linalg.inv(OracleBasis(moved).onee("S"))
    T1, M1 = og.targets(mol, D1)
    T2, M2 = og.targets(moved, D2)
    assert np.array_equal(M1, M2)
    assert np.abs(T1 - T2).max() < 1e-9 * np.abs(T1).max()
    # and the matrix itself is not invariant (the test has teeth)
    assert np.abs(D1 - D2).max() > 1e-2 * np.abs(D1).max()


def test_assembly_undoes_the_local_transform(dimer_pair):
    mol, _ = dimer_pair
    rng = np.random.default_rng(3)
    N = og.atom_layout(mol)[1]
    D = rng.standard_normal((N, N))
    D = D + D.T
    T, M = og.targets(mol, D)
    assert np.abs(og.assemble(mol, T) - D).max() < 1e-11
