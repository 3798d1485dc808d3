"""Real solid-harmonic (spherical) basis on the oracle side -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the benchmark's CPU leg may import this.

Paper Sec. 2.1.1: contracted functions are real solid harmonics times
Gaussians.  The oracle builds the spherical functions of each shell from the
defining polynomials of the real solid harmonics,
    l = 0: 1;  l = 1: x, y, z;
    l = 2: xy, yz, 2z^2 - x^2 - y^2, xz, x^2 - y^2   (m = -2 .. 2),
    l = 3: y(3x^2 - y^2), xyz, y(4z^2 - x^2 - y^2), z(2z^2 - 3x^2 - 3y^2),
           x(4z^2 - x^2 - y^2), z(x^2 - y^2), x(x^2 - 3y^2)   (m = -3 .. 3),
written on its own unit-normalised Cartesian functions (a monomial x^i y^j z^k
is its normalised component times sqrt((2i-1)!!(2j-1)!!(2k-1)!!) up to a
common factor), and then rescales each spherical function to unit norm with
its own overlap matrix.  Orthogonality within a shell is not imposed; the
pins check that it comes out.  Every spherical matrix is then the plain
change of basis of the Cartesian one: M = T M_cart T^T, and J, K of a
spherical density D are T J_cart[T^T D T] T^T (the ERIs transform with T on
every index, and J, K are linear in them and in D).
"""
from __future__ import annotations

import numpy as np

from .oracle import OracleBasis

_POLY = {
    0: [{(0, 0, 0): 1.0}],
    1: [{(1, 0, 0): 1.0}, {(0, 1, 0): 1.0}, {(0, 0, 1): 1.0}],
    2: [{(1, 1, 0): 1.0}, {(0, 1, 1): 1.0}, {(0, 0, 2): 2.0, (2, 0, 0): -1.0, (0, 2, 0): -1.0},
        {(1, 0, 1): 1.0}, {(2, 0, 0): 1.0, (0, 2, 0): -1.0}],
    3: [{(2, 1, 0): 3.0, (0, 3, 0): -1.0}, {(1, 1, 1): 1.0},
        {(0, 1, 2): 4.0, (2, 1, 0): -1.0, (0, 3, 0): -1.0},
        {(0, 0, 3): 2.0, (2, 0, 1): -3.0, (0, 2, 1): -3.0},
        {(1, 0, 2): 4.0, (3, 0, 0): -1.0, (1, 2, 0): -1.0},
        {(2, 0, 1): 1.0, (0, 2, 1): -1.0}, {(3, 0, 0): 1.0, (1, 2, 0): -3.0}],
}


def _cart_components(l):
    """(i, j, k) of the Cartesian components in the engine's order (x-major, descending)."""
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def _dfact(n):
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


class SphericalOracleBasis:
    """Spherical view of an OracleBasis: nbf spherical functions, T (nbf x nbf_cart)."""

    def __init__(self, mol):
        self.cart = OracleBasis(mol)
        self.mol = mol
        S = self.cart.onee("S")
        rows = []
        for s, l in enumerate(self.cart.shell_l):
            l = int(l)
            comps = _cart_components(l)
            a0 = int(self.cart.ao[s])
            for poly in _POLY[l]:
                t = np.zeros(self.cart.nbf)
                for (i, j, k), c in poly.items():
                    t[a0 + comps.index((i, j, k))] = c * np.sqrt(_dfact(2 * i - 1) * _dfact(2 * j - 1) * _dfact(2 * k - 1))
                t /= np.sqrt(t @ S @ t)
                rows.append(t)
        self.T = np.array(rows)
        self.nbf = self.T.shape[0]
        self.nbf_cart = self.cart.nbf

    def onee(self, which: str) -> np.ndarray:
        return self.T @ self.cart.onee(which) @ self.T.T

    def enuc(self) -> float:
        return self.cart.enuc()

    def jk(self, D: np.ndarray, tau: float = 0.0, nthreads: int = 0):
        Dc = self.T.T @ np.asarray(D, dtype=np.float64) @ self.T
        Jc, Kc, nq = self.cart.jk(Dc, tau=tau, nthreads=nthreads)
        return self.T @ Jc @ self.T.T, self.T @ Kc @ self.T.T, nq
