"""Plain numpy restatement of the learned initial density's geometry.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no
learned guess; the definitions restated here are this project's reading of
the task's learned-guess configuration (a network maps per-atom-pair
geometric features to density blocks):

* pair frame (A, B), A <= B: z along A -> B; x towards the atom nearest to the
  pair's midpoint, made perpendicular to z; y = z x x.  Self pair (A, A): z
  towards the nearest neighbour of A, x towards the second nearest.  Rows of
  the frame matrix R are the local x, y, z axes in global coordinates.
* features (48 per pair): r_AB / 10; one-hot element of A and of B (H, C, N,
  O); 32 Gaussian radial basis values of r_AB (centres 10 k / 31 bohr, width
  0.4); distances / 10 of the frame atom(s) to A and B (self pairs: of the
  two neighbours to A); one-hot element of the frame atom C; self flag.
* shell transform U under a rotation R: the normalised Cartesian functions
  g_c (monomial times its component normalisation, so xx carries 1/sqrt(3)
  against xy) obey g(R v) = U g(v).  U is found here by least squares over
  sampled points, not from a closed form.
* local block L = U_A^{-T} D_AB U_B^{-1}; assembly D_AB = U_A^T L U_B (self
  blocks symmetrised), both halves of D written.

Parity unpinned by the paper (it has no learned guess): the pins are the
rotation covariance of the blocks, the invariance of the features, the
round trip, and hand-worked rotations (tests/test_oracle_pins_guess.py).
"""
from __future__ import annotations

import math

import numpy as np

NFEAT = 48
MAXF = 15
NOUT = MAXF * MAXF
_ELEM = {1: 0, 6: 1, 7: 2, 8: 3}


def cart_components(l: int):
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


def _dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def _g(l: int, v: np.ndarray) -> np.ndarray:
    """Normalised Cartesian functions of one shell at points v (k x 3): (ncart, k)."""
    out = []
    for c in cart_components(l):
        n = 1.0 / math.sqrt(_dfact(2 * c[0] - 1) * _dfact(2 * c[1] - 1) * _dfact(2 * c[2] - 1))
        out.append(n * v[:, 0] ** c[0] * v[:, 1] ** c[1] * v[:, 2] ** c[2])
    return np.array(out)


def shell_U(l: int, R: np.ndarray) -> np.ndarray:
    """U with g(R v) = U g(v), by least squares over 40 seeded points."""
    v = np.random.default_rng(12345).standard_normal((40, 3))
    G = _g(l, v)
    Grot = _g(l, v @ R.T)
    U, *_ = np.linalg.lstsq(G.T, Grot.T, rcond=None)
    return U.T


def atom_U(shell_ls, R) -> np.ndarray:
    n = sum((l + 1) * (l + 2) // 2 for l in shell_ls)
    U = np.zeros((n, n))
    off = 0
    for l in shell_ls:
        k = (l + 1) * (l + 2) // 2
        U[off:off + k, off:off + k] = shell_U(l, R)
        off += k
    return U


def frame(z, hint) -> np.ndarray:
    z = np.asarray(z, float) / np.linalg.norm(z)
    x = np.asarray(hint, float) - np.dot(hint, z) * z
    if not np.linalg.norm(x) > 1e-6:
        e = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        x = e - np.dot(e, z) * z
    x = x / np.linalg.norm(x)
    return np.array([x, np.cross(z, x), z])


def pairs(mol):
    """[(A, B, R, features)] for A <= B in the library's pair order."""
    X = np.asarray(mol.xyz, float)
    Z = list(mol.Z)
    na = len(Z)
    out = []
    for A in range(na):
        for B in range(A, na):
            f = np.zeros(NFEAT)
            others = [c for c in range(na) if c != A and c != B]
            if A != B:
                zv = X[B] - X[A]
                r = float(np.linalg.norm(zv))
                mid = 0.5 * (X[A] + X[B])
                if others:
                    d = [np.linalg.norm(X[c] - mid) for c in others]
                    C = others[int(np.argmin(d))]
                    R = frame(zv, X[C] - mid)
                    f[41], f[42] = 0.1 * np.linalg.norm(X[C] - X[A]), 0.1 * np.linalg.norm(X[C] - X[B])
                    if Z[C] in _ELEM:
                        f[43 + _ELEM[Z[C]]] = 1.0
                else:
                    R = frame(zv, np.zeros(3))
            else:
                r = 0.0
                d = np.array([np.linalg.norm(X[c] - X[A]) for c in others])
                order = [others[i] for i in np.argsort(d, kind="stable")]
                zv = X[order[0]] - X[A] if order else np.array([0.0, 0.0, 1.0])
                hint = X[order[1]] - X[A] if len(order) > 1 else np.zeros(3)
                R = frame(zv, hint)
                if order:
                    f[41] = 0.1 * np.linalg.norm(X[order[0]] - X[A])
                    if Z[order[0]] in _ELEM:
                        f[43 + _ELEM[Z[order[0]]]] = 1.0
                if len(order) > 1:
                    f[42] = 0.1 * np.linalg.norm(X[order[1]] - X[A])
                f[47] = 1.0
            f[0] = 0.1 * r
            if Z[A] in _ELEM:
                f[1 + _ELEM[Z[A]]] = 1.0
            if Z[B] in _ELEM:
                f[5 + _ELEM[Z[B]]] = 1.0
            mu = 10.0 * np.arange(32) / 31.0
            f[9:41] = np.exp(-(r - mu) ** 2 / (2 * 0.4 ** 2))
            out.append((A, B, R, f))
    return out


def atom_layout(mol):
    """(first function, shell l list) per atom, shells of an atom contiguous."""
    first, ls, off = {}, {}, 0
    for s in mol.shells:
        first.setdefault(s.atom, off)
        ls.setdefault(s.atom, []).append(s.l)
        off += (s.l + 1) * (s.l + 2) // 2
    return [(first[a], ls[a]) for a in range(len(mol.Z))], off


def features(mol) -> np.ndarray:
    return np.array([p[3] for p in pairs(mol)])


def targets(mol, D):
    """Local blocks L (npairs x 225, row-major 15 x 15 padding) and their mask."""
    lay, _ = atom_layout(mol)
    T = np.zeros((len(pairs(mol)), NOUT))
    M = np.zeros_like(T)
    for p, (A, B, R, _) in enumerate(pairs(mol)):
        (fa, la), (fb, lb) = lay[A], lay[B]
        UA, UB = atom_U(la, R), atom_U(lb, R)
        na, nb = UA.shape[0], UB.shape[0]
        L = np.linalg.inv(UA).T @ D[fa:fa + na, fb:fb + nb] @ np.linalg.inv(UB)
        blk = np.zeros((MAXF, MAXF))
        blk[:na, :nb] = L
        msk = np.zeros((MAXF, MAXF))
        msk[:na, :nb] = 1.0
        T[p], M[p] = blk.ravel(), msk.ravel()
    return T, M


def assemble(mol, blocks) -> np.ndarray:
    """D from local blocks (npairs x 225): D_AB = U_A^T L U_B, self blocks symmetrised."""
    lay, N = atom_layout(mol)
    D = np.zeros((N, N))
    for p, (A, B, R, _) in enumerate(pairs(mol)):
        (fa, la), (fb, lb) = lay[A], lay[B]
        UA, UB = atom_U(la, R), atom_U(lb, R)
        na, nb = UA.shape[0], UB.shape[0]
        L = np.asarray(blocks[p], float).reshape(MAXF, MAXF)[:na, :nb]
        blk = UA.T @ L @ UB
        if A == B:
            blk = 0.5 * (blk + blk.T)
        D[fa:fa + na, fb:fb + nb] = blk
        D[fb:fb + nb, fa:fa + na] = blk.T
    return D
