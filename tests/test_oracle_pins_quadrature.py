"""More pins of the CPU oracle, each by a route that shares nothing with it.

* One-electron integrals of p and d shells (Sec. 2.3.1-2.3.3, Eqs. s-overall,
  Tab-final, Vab-final) against Gauss-Hermite quadrature of their defining
  integrals: the overlap as the integral of the polynomial times the Gaussian
  product; the kinetic energy with the ket's second derivative written out
  analytically; the nuclear attraction through the Gaussian transform
  1/r_C = (2/sqrt(pi)) int_0^inf exp(-u^2 r_C^2) du, whose u-integral is done
  by Gauss-Legendre.  No Hermite expansion coefficient, Hermite Coulomb
  integral or Boys function appears on this side.
* The by-definition J/K block (Eq. fock over every ordered ket shell pair,
  used to check sampled blocks of large molecules) against the brute-force
  contraction of the full ERI tensor and against the unique-quartet build.
"""
import math
from itertools import product

import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss

from fsim_synth import workload
from oracle import OracleBasis

from .gauss_transform import cart_components, contracted_coefs
from .helpers import make_mol, random_mol

pytestmark = pytest.mark.filterwarnings("ignore")

_ZH, _WH = hermgauss(12)           # exact for polynomials of degree <= 23
_TL, _WL = leggauss(96)
_TL, _WL = 0.5 * (_TL + 1.0), 0.5 * _WL


def _axis_moments(i, j, a, b, A, B, g_extra=0.0, C=0.0):
    """int (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2 - g_extra (x-C)^2) dx and the
    same integral with the ket's -1/2 d^2/dx^2 applied to (x-B)^j exp(-b(x-B)^2).
    g_extra may be an array (one value per u-node); so is the result."""
    g_extra = np.asarray(g_extra, dtype=float)
    p = a + b + g_extra
    S = (a * A + b * B + g_extra * C) / p
    # the three Gaussians combine into exp(-p (x-S)^2) times a constant
    c0 = a * A * A + b * B * B + g_extra * C * C - p * S * S
    x = S[..., None] + _ZH / np.sqrt(p)[..., None]
    pref = np.exp(-c0) / np.sqrt(p)
    xa, xb = x - A, x - B
    s = pref * ((xa ** i * xb ** j) @ _WH)
    d2 = -2.0 * b * (2 * j + 1) * xb ** j + 4.0 * b * b * xb ** (j + 2)
    if j >= 2:
        d2 = d2 + j * (j - 1) * xb ** (j - 2)
    t = pref * ((-0.5 * xa ** i * d2) @ _WH)
    return s, t


def _quadrature_onee(mol):
    """S, T, V over the normalised contracted Cartesian basis, by quadrature."""
    shells = mol.shells
    comps = [cart_components(s.l) for s in shells]
    ao = np.cumsum([0] + [len(c) for c in comps])
    N = int(ao[-1])
    S, T, V = np.zeros((N, N)), np.zeros((N, N)), np.zeros((N, N))
    for sa, sb in product(range(len(shells)), repeat=2):
        A, B = mol.xyz[shells[sa].atom], mol.xyz[shells[sb].atom]
        ca = np.array([contracted_coefs(shells[sa].l, shells[sa].alpha, shells[sa].coef, c) for c in comps[sa]])
        cb = np.array([contracted_coefs(shells[sb].l, shells[sb].alpha, shells[sb].coef, c) for c in comps[sb]])
        for ka, a in enumerate(shells[sa].alpha):
            for kb, b in enumerate(shells[sb].alpha):
                p = a + b
                for (ia, i3), (ib, j3) in product(enumerate(comps[sa]), enumerate(comps[sb])):
                    w = ca[ia, ka] * cb[ib, kb]
                    st = [_axis_moments(i3[d], j3[d], a, b, A[d], B[d]) for d in range(3)]
                    s3 = st[0][0] * st[1][0] * st[2][0]
                    t3 = st[0][1] * st[1][0] * st[2][0] + st[0][0] * st[1][1] * st[2][0] \
                        + st[0][0] * st[1][0] * st[2][1]
                    # nuclear attraction: u^2 = p t^2 / (1 - t^2), du = sqrt(p) (1-t^2)^{-3/2} dt
                    u2 = p * _TL * _TL / (1.0 - _TL * _TL)
                    du = math.sqrt(p) * (1.0 - _TL * _TL) ** -1.5 * _WL
                    v = 0.0
                    for Zc, C in zip(mol.Z, mol.xyz):
                        f = np.ones_like(_TL)
                        for d in range(3):
                            f = f * _axis_moments(i3[d], j3[d], a, b, A[d], B[d], u2, C[d])[0]
                        v += -Zc * 2.0 / math.sqrt(math.pi) * float(np.sum(f * du))
                    r, c = ao[sa] + ia, ao[sb] + ib
                    S[r, c] += w * s3
                    T[r, c] += w * t3
                    V[r, c] += w * v
    return S, T, V


def _spd_mol(seed):
    # two or three atoms with s, p and d shells of 2 primitives, plus one 3-primitive d shell
    rng = np.random.default_rng(seed)
    m = random_mol(rng, natom=2, lmax=2, nprim=2, spread=1.2)
    extra = (1, 2, (0.35, 0.9, 2.2), (0.5, 0.8, 0.3))
    return make_mol([(int(z), tuple(x)) for z, x in zip(m.Z, m.xyz)],
                    [(s.atom, s.l, s.alpha, s.coef) for s in m.shells] + [extra])


def _spdf_mol(seed):
    # the s/p/d molecule plus a 2-primitive f shell on the first atom
    m = _spd_mol(seed)
    return make_mol([(int(z), tuple(x)) for z, x in zip(m.Z, m.xyz)],
                    [(s.atom, s.l, s.alpha, s.coef) for s in m.shells] + [(0, 3, (0.45, 1.3), (0.7, 0.4))])


@pytest.mark.parametrize("seed,f", [(3, False), (17, False), (5, True)])
def test_pd_one_electron_vs_quadrature(seed, f):
    m = _spdf_mol(seed) if f else _spd_mol(seed)
    B = OracleBasis(m)
    Sq, Tq, Vq = _quadrature_onee(m)
    for name, got, ref in (("S", B.onee("S"), Sq), ("T", B.onee("T"), Tq), ("V", B.onee("V"), Vq)):
        err = np.abs(got - ref).max()
        assert err <= 1e-12 * max(1.0, np.abs(ref).max()), (name, err)


def test_jk_block_equals_brute_force_water():
    m = workload("water")
    B = OracleBasis(m)
    g = B.eri_full()
    rng = np.random.default_rng(21)
    D = rng.standard_normal((B.nbf, B.nbf))
    D = D + D.T
    Jref = np.einsum("pqrs,rs->pq", g, D)
    Kref = np.einsum("prqs,rs->pq", g, D)
    for sa, sb in product(range(m.nshell), repeat=2):
        Jb, Kb = B.jk_block(D, sa, sb)
        ra = slice(B.ao[sa], B.ao[sa] + Jb.shape[0])
        rb = slice(B.ao[sb], B.ao[sb] + Jb.shape[1])
        assert np.abs(Jb - Jref[ra, rb]).max() < 1e-12
        assert np.abs(Kb - Kref[ra, rb]).max() < 1e-12


@pytest.mark.parametrize("tau", [0.0, 1e-10, 1e-3])
def test_jk_block_equals_unique_quartet_build(tau):
    # random s/p/d molecule (d shells reach (dd|dd)), every block of J and K
    m = random_mol(np.random.default_rng(8), natom=3, lmax=2, nprim=2, spread=2.5)
    B = OracleBasis(m)
    rng = np.random.default_rng(22)
    D = rng.standard_normal((B.nbf, B.nbf))
    D = D + D.T
    J, K, nq = B.jk(D, tau=tau)
    ns = m.nshell
    if tau >= 1e-3:
        assert nq < ns * (ns + 1) // 2 * (ns * (ns + 1) // 2 + 1) // 2  # screening bites
    Q = B.schwarz() if tau > 0 else None
    scale = max(1.0, np.abs(J).max(), np.abs(K).max())
    for sa, sb in product(range(ns), repeat=2):
        Jb, Kb = B.jk_block(D, sa, sb, tau=tau, Q=Q)
        ra = slice(B.ao[sa], B.ao[sa] + Jb.shape[0])
        rb = slice(B.ao[sb], B.ao[sb] + Jb.shape[1])
        assert np.abs(Jb - J[ra, rb]).max() <= 1e-12 * scale
        assert np.abs(Kb - K[ra, rb]).max() <= 1e-12 * scale
