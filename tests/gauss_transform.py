"""Independent route to two-electron integrals, used only to pin the oracle.

1/r12 = (2/sqrt(pi)) int_0^inf exp(-u^2 r12^2) du.  For fixed u the six-fold
integral over Cartesian Gaussians factorises into three two-dimensional
polynomial-times-Gaussian integrals (x1, x2 per axis).  Each is done exactly
by a Cholesky change of variables and tensor Gauss-Hermite quadrature; the
u-integral is mapped to t in [0, 1) with u^2 = rho t^2 / (1 - t^2),
rho = pq/(p+q), and done by Gauss-Legendre.  Nothing here uses Hermite
expansion coefficients, Hermite Coulomb integrals or the Boys function, so it
checks those parts of the oracle from outside.  Normalisation is restated here
from its closed forms.
"""
from __future__ import annotations

import math
from itertools import product

import numpy as np
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss


def cart_components(l: int) -> list:
    return [(a, b, l - a - b) for a in range(l, -1, -1) for b in range(l - a, -1, -1)]


def dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def prim_norm(alpha: float, comp) -> float:
    l = sum(comp)
    return ((2 * alpha / math.pi) ** 0.75 * (4 * alpha) ** (l / 2)
            / math.sqrt(dfact(2 * comp[0] - 1) * dfact(2 * comp[1] - 1) * dfact(2 * comp[2] - 1)))


def contracted_coefs(l: int, alphas, coefs, comp) -> np.ndarray:
    """d_k N_k for one component, rescaled to unit norm with the closed-form
    overlap of two normalised same-centre primitives (2 sqrt(ab)/(a+b))^(l+3/2)."""
    d = np.array([c * prim_norm(a, comp) for a, c in zip(alphas, coefs)])
    raw = np.array(coefs, dtype=float)
    S = 0.0
    for i, a in enumerate(alphas):
        for j, b in enumerate(alphas):
            S += raw[i] * raw[j] * (2 * math.sqrt(a * b) / (a + b)) ** (l + 1.5)
    return d / math.sqrt(S)


class _Axis2D:
    """Tables I[i][j][k][l](t) for one axis at all u-nodes."""

    def __init__(self, A, B, Cc, D, a, b, c, d, u2, lmax4, zx, wz):
        p, q = a + b, c + d
        P, Q = (a * A + b * B) / p, (c * Cc + d * D) / q
        m11, m22, m12 = p + u2, q + u2, -u2
        det = m11 * m22 - m12 * m12
        # mean m = M^{-1} (pP, qQ)
        r1, r2 = p * P, q * Q
        mu1 = (m22 * r1 - m12 * r2) / det
        mu2 = (-m12 * r1 + m11 * r2) / det
        c0 = p * (mu1 - P) ** 2 + q * (mu2 - Q) ** 2 + u2 * (mu1 - mu2) ** 2
        # Cholesky M = L L^T, L lower: [[l11, 0], [l21, l22]]
        l11 = np.sqrt(m11)
        l21 = m12 / l11
        l22 = np.sqrt(m22 - l21 * l21)
        # y = m + L^{-T} z ; L^{-T} = [[1/l11, -l21/(l11 l22)], [0, 1/l22]]
        z1, z2 = zx[:, 0][None, :], zx[:, 1][None, :]
        y1 = mu1[:, None] + z1 / l11[:, None] - (l21 / (l11 * l22))[:, None] * z2
        y2 = mu2[:, None] + z2 / l22[:, None]
        pref = np.exp(-c0) / (l11 * l22)
        e_ab = math.exp(-a * b / p * (A - B) ** 2)
        e_cd = math.exp(-c * d / q * (Cc - D) ** 2)
        self.tab = {}
        xa, xb, xc, xd = y1 - A, y1 - B, y2 - Cc, y2 - D
        for i, j, k, l in product(*(range(x + 1) for x in lmax4)):
            poly = xa ** i * xb ** j * xc ** k * xd ** l
            # exp(-a (x-A)^2 - b (x-B)^2) = e_ab exp(-p (x-P)^2), same for cd
            self.tab[(i, j, k, l)] = e_ab * e_cd * pref * (poly @ wz)


def prim_block(la, lb, lc, ld, A, B, Cc, D, a, b, c, d, n_gh=8, n_gl=160) -> np.ndarray:
    """[ab|cd] for unnormalised primitives, all Cartesian components."""
    A, B, Cc, D = (np.asarray(v, dtype=float) for v in (A, B, Cc, D))
    p, q = a + b, c + d
    rho = p * q / (p + q)
    x, w = leggauss(n_gl)
    t = 0.5 * (x + 1.0)
    wt = 0.5 * w
    u2 = rho * t * t / (1.0 - t * t)
    du = math.sqrt(rho) * (1.0 - t * t) ** -1.5 * wt
    zh, wh = hermgauss(n_gh)
    Z1, Z2 = np.meshgrid(zh, zh, indexing="ij")
    zx = np.stack([Z1.ravel(), Z2.ravel()], axis=1)
    wz = np.outer(wh, wh).ravel()
    axes = [_Axis2D(A[k], B[k], Cc[k], D[k], a, b, c, d, u2, (la, lb, lc, ld), zx, wz) for k in range(3)]
    ca, cb, cc, cd = (cart_components(l) for l in (la, lb, lc, ld))
    out = np.zeros((len(ca), len(cb), len(cc), len(cd)))
    for (ia, i3), (ib, j3), (ic, k3), (id_, l3) in product(enumerate(ca), enumerate(cb),
                                                            enumerate(cc), enumerate(cd)):
        f = np.ones_like(t)
        for k in range(3):
            f = f * axes[k].tab[(i3[k], j3[k], k3[k], l3[k])]
        out[ia, ib, ic, id_] = 2.0 / math.sqrt(math.pi) * float(np.sum(f * du))
    return out


def contracted_block(shells, centres) -> np.ndarray:
    """(ab|cd) for four contracted shells given as (l, alphas, coefs)."""
    ls = [s[0] for s in shells]
    comps = [cart_components(l) for l in ls]
    cn = [np.array([contracted_coefs(s[0], s[1], s[2], c) for c in comps[n]]) for n, s in enumerate(shells)]
    out = np.zeros([len(c) for c in comps])
    for k0, k1, k2, k3 in product(*(range(len(s[1])) for s in shells)):
        blk = prim_block(*ls, *centres, shells[0][1][k0], shells[1][1][k1], shells[2][1][k2], shells[3][1][k3])
        w = np.einsum("a,b,c,d->abcd", cn[0][:, k0], cn[1][:, k1], cn[2][:, k2], cn[3][:, k3])
        out += w * blk
    return out
