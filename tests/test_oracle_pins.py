"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: closed forms, quadrature of a
definition, an independent integral route (tests/gauss_transform.py),
finite differences, symmetry, positivity, invariance and SCF invariants.
"""
import math

import numpy as np
import pytest
from numpy.polynomial.hermite import hermgauss
from numpy.polynomial.legendre import leggauss

from fsim_synth import workload
from oracle import OracleBasis, boys, hermite_E, hermite_R, jacobi_eigh, rhf
from oracle.scf import orthogonaliser

from .gauss_transform import contracted_block, prim_block, cart_components
from .helpers import make_mol, random_mol

pytestmark = pytest.mark.filterwarnings("ignore")


# ---------------------------------------------------------------- Boys (Sec. 2.3.3)
@pytest.mark.parametrize("n", range(0, 17))
def test_boys_at_zero(n):
    # F_n(0) = int_0^1 t^{2n} dt = 1/(2n+1)
    assert boys(n, 0.0) == pytest.approx(1.0 / (2 * n + 1), rel=1e-15)


@pytest.mark.parametrize("T", [1e-6, 0.01, 0.3, 1.0, 4.7, 12.0, 29.9, 39.99, 40.0, 55.0, 120.0])
def test_boys_f0_erf(T):
    # F_0(T) = (1/2) sqrt(pi/T) erf(sqrt T)
    ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert boys(0, T) == pytest.approx(ref, rel=2e-14)


@pytest.mark.parametrize("n", [0, 1, 3, 5, 8, 12])
@pytest.mark.parametrize("T", [0.05, 0.9, 3.3, 11.0, 25.0, 38.0, 45.0, 70.0])
def test_boys_quadrature(n, T):
    # Gauss-Legendre on the definition int_0^1 exp(-T t^2) t^{2n} dt
    x, w = leggauss(200)
    t = 0.5 * (x + 1)
    ref = 0.5 * float(np.sum(w * np.exp(-T * t * t) * t ** (2 * n)))
    assert boys(n, T) == pytest.approx(ref, rel=1e-13)


@pytest.mark.parametrize("T", [0.2, 7.5, 39.9, 40.1, 80.0])
def test_boys_downward_identity(T):
    # F_n = (2T F_{n+1} + exp(-T)) / (2n+1), integration by parts of the definition
    for n in range(0, 12):
        lhs = boys(n, T)
        rhs = (2 * T * boys(n + 1, T) + math.exp(-T)) / (2 * n + 1)
        assert lhs == pytest.approx(rhs, rel=1e-13)


# ---------------------------------------------------------------- E coefficients (Sec. 2.1.3)
def _hermite_gaussian(t, p, xP):
    # Lambda_t = (d/dP)^t exp(-p x_P^2) = p^{t/2} H_t(sqrt(p) x_P) exp(-p x_P^2)
    Ht = np.polynomial.hermite.hermval(math.sqrt(p) * xP, [0] * t + [1])
    return p ** (t / 2) * Ht * np.exp(-p * xP * xP)


@pytest.mark.parametrize("i,j", [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (2, 1), (2, 2), (0, 2), (1, 2)])
def test_hermite_expansion_pointwise(i, j):
    # (x-A)^i (x-B)^j exp(-a(x-A)^2 - b(x-B)^2) = sum_t E^{ij}_t Lambda_t(x_P)
    a, b, A, B = 0.7, 1.9, 0.3, -0.45
    p = a + b
    P = (a * A + b * B) / p
    x = np.linspace(-3, 3, 41)
    lhs = (x - A) ** i * (x - B) ** j * np.exp(-a * (x - A) ** 2 - b * (x - B) ** 2)
    rhs = sum(hermite_E(i, j, t, A - B, a, b) * _hermite_gaussian(t, p, x - P) for t in range(i + j + 1))
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-14)
    assert hermite_E(i, j, -1, A - B, a, b) == 0.0
    assert hermite_E(i, j, i + j + 1, A - B, a, b) == 0.0


def test_e00_and_overlap_axis():
    # E^{00}_0 = exp(-mu X^2) and S_ij = E^{ij}_0 sqrt(pi/p) (Eq. sx-final) vs Gauss-Hermite
    a, b, A, B = 0.35, 1.1, 1.2, -0.4
    p, mu = a + b, a * b / (a + b)
    assert hermite_E(0, 0, 0, A - B, a, b) == pytest.approx(math.exp(-mu * (A - B) ** 2), rel=1e-15)
    z, w = hermgauss(20)
    P = (a * A + b * B) / p
    x = P + z / math.sqrt(p)
    for i in range(3):
        for j in range(3):
            ref = math.exp(-mu * (A - B) ** 2) / math.sqrt(p) * float(np.sum(w * (x - A) ** i * (x - B) ** j))
            assert hermite_E(i, j, 0, A - B, a, b) * math.sqrt(math.pi / p) == pytest.approx(ref, rel=1e-13, abs=1e-16)


# ---------------------------------------------------------------- R (Sec. 2.3.3)
def test_hermite_R_is_derivative_of_boys():
    # R^0_tuv = d^t/dX d^u/dY d^v/dZ F_0(a |R|^2)  (Eq. Rn-definition, n = 0), by central differences
    a, X, Y, Z = 0.9, 0.4, -0.7, 1.1
    f = lambda x, y, z: boys(0, a * (x * x + y * y + z * z))
    h = 1e-3
    d1 = (f(X + h, Y, Z) - f(X - h, Y, Z)) / (2 * h)
    assert hermite_R(0, 1, 0, 0, a, X, Y, Z) == pytest.approx(d1, rel=1e-6)
    d2 = (f(X, Y + h, Z) - 2 * f(X, Y, Z) + f(X, Y - h, Z)) / h ** 2
    assert hermite_R(0, 0, 2, 0, a, X, Y, Z) == pytest.approx(d2, rel=1e-5)
    dxz = (f(X + h, Y, Z + h) - f(X + h, Y, Z - h) - f(X - h, Y, Z + h) + f(X - h, Y, Z - h)) / (4 * h * h)
    assert hermite_R(0, 1, 0, 1, a, X, Y, Z) == pytest.approx(dxz, rel=1e-5)
    # source term R^n_000 = (-2a)^n F_n(a R^2)
    T = a * (X * X + Y * Y + Z * Z)
    assert hermite_R(3, 0, 0, 0, a, X, Y, Z) == pytest.approx((-2 * a) ** 3 * boys(3, T), rel=1e-15)


# ---------------------------------------------------------------- one-electron (Sec. 2.3.1-2.3.3)
def _two_s(a, b, R, ZA=1, ZB=1):
    return make_mol([(ZA, (0, 0, 0)), (ZB, (0.3, -0.2, R))],
                    [(0, 0, (a,), (1.0,)), (1, 0, (b,), (1.0,))], "two_s")


@pytest.mark.parametrize("a,b,R", [(0.5, 0.5, 1.4), (0.3, 1.7, 0.8), (2.2, 0.15, 3.0)])
def test_ss_one_electron_closed_forms(a, b, R):
    m = _two_s(a, b, R, 3, 1)
    B = OracleBasis(m)
    S, T, V = B.onee("S"), B.onee("T"), B.onee("V")
    A, Bc = m.xyz[0], m.xyz[1]
    p, mu = a + b, a * b / (a + b)
    R2 = float(np.sum((A - Bc) ** 2))
    Na, Nb = (2 * a / math.pi) ** 0.75, (2 * b / math.pi) ** 0.75
    s = (math.pi / p) ** 1.5 * math.exp(-mu * R2)
    assert np.allclose(np.diag(S), 1.0, atol=1e-14)
    assert S[0, 1] == pytest.approx(Na * Nb * s, rel=1e-13)
    assert T[0, 1] == pytest.approx(Na * Nb * mu * (3 - 2 * mu * R2) * s, rel=1e-12)
    P = (a * A + b * Bc) / p
    v = 0.0
    for Zc, C in zip(m.Z, m.xyz):
        RPC2 = float(np.sum((P - C) ** 2))
        # F_0 by its erf closed form
        F0 = 1.0 if RPC2 == 0 else 0.5 * math.sqrt(math.pi / (p * RPC2)) * math.erf(math.sqrt(p * RPC2))
        v += -Zc * 2 * math.pi / p * math.exp(-mu * R2) * F0
    assert V[0, 1] == pytest.approx(Na * Nb * v, rel=1e-12)


def test_kinetic_symmetric_positive_definite():
    # -1/2 Laplacian is a positive operator: T is symmetric positive definite for any basis
    m = random_mol(np.random.default_rng(5), natom=2, lmax=2, nprim=2)
    B = OracleBasis(m)
    T = B.onee("T")
    assert np.allclose(T, T.T, atol=1e-13)
    assert np.linalg.eigvalsh(T).min() > 0


def test_onee_translation_invariance():
    rng = np.random.default_rng(11)
    m = random_mol(rng, natom=2, lmax=2, nprim=2)
    m2 = make_mol([(z, tuple(x + np.array([1.3, -0.7, 2.1]))) for z, x in zip(m.Z, m.xyz)],
                  [(s.atom, s.l, s.alpha, s.coef) for s in m.shells])
    for w in "STV":
        assert np.allclose(OracleBasis(m).onee(w), OracleBasis(m2).onee(w), atol=1e-12)


# ---------------------------------------------------------------- ERIs (Sec. 2.3.4)
@pytest.mark.parametrize("a,b,c,d", [(0.5, 0.5, 0.5, 0.5), (0.3, 1.9, 0.8, 0.2), (2.5, 2.0, 0.12, 0.4)])
def test_ssss_closed_form(a, b, c, d):
    # (ss|ss) = 2 pi^{5/2} / (pq sqrt(p+q)) K_AB K_CD F_0(alpha R_PQ^2), F_0 via erf
    cen = [np.array(v) for v in [(0, 0, 0), (0.4, 0.1, -0.9), (1.3, -0.6, 0.2), (-0.8, 1.0, 0.6)]]
    m = make_mol([(1, tuple(v)) for v in cen], [(i, 0, (x,), (1.0,)) for i, x in enumerate((a, b, c, d))])
    B = OracleBasis(m)
    v = B.eri_block(0, 1, 2, 3)[0, 0, 0, 0]
    p, q = a + b, c + d
    P, Q = (a * cen[0] + b * cen[1]) / p, (c * cen[2] + d * cen[3]) / q
    al = p * q / (p + q)
    T = al * float(np.sum((P - Q) ** 2))
    F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-a * b / p * np.sum((cen[0] - cen[1]) ** 2)) \
        * math.exp(-c * d / q * np.sum((cen[2] - cen[3]) ** 2)) * F0
    N = np.prod([(2 * x / math.pi) ** 0.75 for x in (a, b, c, d)])
    assert v == pytest.approx(N * ref, rel=1e-13)


CLASSES = [(1, 0, 0, 0), (1, 1, 0, 0), (1, 0, 1, 0), (1, 1, 1, 1), (2, 0, 0, 0), (2, 1, 0, 0),
           (2, 0, 2, 0), (2, 1, 1, 0), (2, 2, 0, 0), (2, 1, 2, 1), (2, 2, 1, 1), (2, 2, 2, 0), (2, 2, 2, 2),
           (0, 2, 1, 2), (1, 2, 0, 1),
           # f shells: every f pair class, f on the ket side, and (ff|ff)
           (3, 0, 0, 0), (3, 1, 0, 0), (3, 2, 1, 0), (3, 3, 0, 0), (1, 0, 3, 2), (3, 1, 3, 1), (3, 3, 3, 3)]


@pytest.mark.parametrize("cls", CLASSES)
def test_eri_class_vs_gaussian_transform(cls):
    # every class against the quadrature route that shares nothing with E, R or Boys
    rng = np.random.default_rng(sum(l * 7 ** i for i, l in enumerate(cls)))
    cen = [tuple(rng.uniform(-1.2, 1.2, 3)) for _ in range(4)]
    al = [float(x) for x in rng.uniform(0.25, 1.6, 4)]
    m = make_mol([(1, c) for c in cen], [(i, cls[i], (al[i],), (1.0,)) for i in range(4)])
    B = OracleBasis(m)
    got = B.eri_block(0, 1, 2, 3)
    raw = prim_block(*cls, *cen, *al)
    comps = [cart_components(l) for l in cls]
    from .gauss_transform import prim_norm
    N = np.einsum("a,b,c,d->abcd", *[np.array([prim_norm(al[i], c) for c in comps[i]]) for i in range(4)])
    ref = N * raw
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_contracted_block_vs_gaussian_transform():
    # contraction + normalisation, (dp|pd) with 2-3 primitives per shell
    shells = [(2, (0.4, 1.0, 2.5), (0.5, 0.7, 0.3)), (1, (0.3, 0.9), (0.6, 0.8)),
              (1, (0.5, 1.25), (0.2, 0.9)), (2, (0.35, 0.875, 2.2), (0.9, 0.4, 0.6))]
    cen = [(0.0, 0.0, 0.0), (0.9, -0.3, 0.4), (-0.5, 1.1, 0.2), (0.3, 0.4, -1.0)]
    m = make_mol([(1, c) for c in cen], [(i, s[0], s[1], s[2]) for i, s in enumerate(shells)])
    got = OracleBasis(m).eri_block(0, 1, 2, 3)
    ref = contracted_block(shells, [np.array(c) for c in cen])
    assert np.abs(got - ref).max() <= 1e-12


def _single_prim_mol(ls, cen, al):
    return make_mol([(1, tuple(c)) for c in cen], [(i, ls[i], (al[i],), (1.0,)) for i in range(4)])


def test_centre_derivative_relation():
    # d/dA_x of a primitive x_A^i exp(-a x_A^2) = 2a (i+1 component) - i (i-1 component)
    # (the derivative relation of Sec. 2.3.2), checked on (p s|s s) from (s s|s s) and (d s|s s)
    cen = [np.array(v) for v in [(0.1, 0.2, -0.3), (0.9, -0.4, 0.5), (-0.7, 0.6, 0.1), (0.4, -0.9, -0.6)]]
    al = [0.8, 0.6, 1.1, 0.45]

    def raw(ls, c):
        B = OracleBasis(_single_prim_mol(ls, c, al))
        from .gauss_transform import prim_norm, cart_components as cc
        comps = [cc(l) for l in ls]
        N = np.einsum("a,b,c,d->abcd", *[np.array([prim_norm(al[i], x) for x in comps[i]]) for i in range(4)])
        return B.eri_block(0, 1, 2, 3) / N

    h = 1e-3
    def shifted(dx):
        c = [v.copy() for v in cen]
        c[0] = c[0] + np.array([dx, 0, 0])
        return raw((0, 0, 0, 0), c)[0, 0, 0, 0]
    # Richardson-extrapolated central difference
    d_h = (shifted(h) - shifted(-h)) / (2 * h)
    d_2h = (shifted(2 * h) - shifted(-2 * h)) / (4 * h)
    deriv = (4 * d_h - d_2h) / 3
    pssss = raw((1, 0, 0, 0), cen)[0, 0, 0, 0]  # x component
    assert deriv == pytest.approx(2 * al[0] * pssss, rel=1e-8)
    # d/dA_x of the p_x primitive: 2a (d_xx) - 1 (s)
    def shifted_p(dx):
        c = [v.copy() for v in cen]
        c[0] = c[0] + np.array([dx, 0, 0])
        return raw((1, 0, 0, 0), c)[0, 0, 0, 0]
    d_h = (shifted_p(h) - shifted_p(-h)) / (2 * h)
    d_2h = (shifted_p(2 * h) - shifted_p(-2 * h)) / (4 * h)
    deriv = (4 * d_h - d_2h) / 3
    dxx = raw((2, 0, 0, 0), cen)[0, 0, 0, 0]
    ssss = raw((0, 0, 0, 0), cen)[0, 0, 0, 0]
    assert deriv == pytest.approx(2 * al[0] * dxx - ssss, rel=1e-8)


@pytest.fixture(scope="module")
def water_full():
    m = workload("water")
    B = OracleBasis(m)
    return m, B, B.eri_full()


def test_eri_eightfold_symmetry(water_full):
    _, _, g = water_full
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.abs(g - g.transpose(perm)).max() < 1e-14


def test_eri_supermatrix_psd_and_schwarz(water_full):
    _, B, g = water_full
    N = B.nbf
    M = g.reshape(N * N, N * N)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > -1e-12
    dg = np.sqrt(np.abs(np.diag(M)))
    assert np.all(np.abs(M) <= np.outer(dg, dg) * (1 + 1e-12) + 1e-15)


def test_eri_rotation_covariance():
    # rotating all centres rotates p blocks by R and d blocks by the induced 6x6 map
    rng = np.random.default_rng(3)
    cen = [rng.uniform(-1, 1, 3) for _ in range(4)]
    al = [0.7, 0.5, 0.9, 0.4]
    ls = (1, 2, 1, 0)
    th = 0.7
    Rm = np.array([[1, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    Rm = Rm @ np.array([[math.cos(0.3), 0, math.sin(0.3)], [0, 1, 0], [-math.sin(0.3), 0, math.cos(0.3)]])
    g0 = OracleBasis(_single_prim_mol(ls, cen, al)).eri_block(0, 1, 2, 3)
    g1 = OracleBasis(_single_prim_mol(ls, [Rm @ c for c in cen], al)).eri_block(0, 1, 2, 3)
    from .gauss_transform import prim_norm
    # transform in unnormalised monomials, then renormalise
    def tmat(l):
        comps = cart_components(l)
        if l == 0:
            return np.ones((1, 1))
        if l == 1:
            return Rm.copy()
        T = np.zeros((6, 6))  # x'_i x'_j = sum R_ik R_jl x_k x_l
        idx = {c: n for n, c in enumerate(comps)}
        for n, c in enumerate(comps):
            i, j = [k for k in range(3) for _ in range(c[k])]
            for k in range(3):
                for l_ in range(3):
                    e = [0, 0, 0]
                    e[k] += 1
                    e[l_] += 1
                    T[n, idx[tuple(e)]] += Rm[i, k] * Rm[j, l_]
        return T
    def unnorm(g, a):
        comps = [cart_components(l) for l in ls]
        N = np.einsum("a,b,c,d->abcd", *[np.array([prim_norm(a[i], x) for x in comps[i]]) for i in range(4)])
        return g / N
    u0, u1 = unnorm(g0, al), unnorm(g1, al)
    pred = np.einsum("ai,bj,ck,dl,ijkl->abcd", tmat(ls[0]), tmat(ls[1]), tmat(ls[2]), tmat(ls[3]), u0)
    assert np.abs(pred - u1).max() < 1e-12


def test_eri_translation_invariance():
    # moving every centre by the same vector leaves every ERI of an s/p/d molecule unchanged
    rng = np.random.default_rng(12)
    m = random_mol(rng, natom=3, lmax=2, nprim=2)
    shift = np.array([2.3, -1.1, 0.6])
    m2 = make_mol([(z, tuple(x + shift)) for z, x in zip(m.Z, m.xyz)],
                  [(s.atom, s.l, s.alpha, s.coef) for s in m.shells])
    B, B2 = OracleBasis(m), OracleBasis(m2)
    ns = m.nshell
    for q in [(0, 1, 2, 3), (2, 2, 5, 5), (8, 5, 2, 7), (3, 4, 6, 8), (5, 8, 8, 2)]:
        q = tuple(x % ns for x in q)
        assert np.abs(B.eri_block(*q) - B2.eri_block(*q)).max() < 1e-12


def test_eri_far_field():
    # separated s distributions: (ab|cd) -> S_ab S_cd / R
    a, b, c, d = 1.0, 1.3, 0.9, 1.1
    for Rz in (40.0, 80.0):
        cen = [(0, 0, 0), (0.3, 0, 0), (0, 0, Rz), (0.2, 0.1, Rz)]
        m = make_mol([(1, x) for x in cen], [(i, 0, (x,), (1.0,)) for i, x in enumerate((a, b, c, d))])
        B = OracleBasis(m)
        S = B.onee("S")
        v = B.eri_block(0, 1, 2, 3)[0, 0, 0, 0]
        P = (a * np.array(cen[0]) + b * np.array(cen[1])) / (a + b)
        Q = (c * np.array(cen[2]) + d * np.array(cen[3])) / (c + d)
        assert v == pytest.approx(S[0, 1] * S[2, 3] / np.linalg.norm(P - Q), rel=1e-12)


# ---------------------------------------------------------------- J / K (Eq. fock)
def test_jk_unique_quartets_equal_brute_force(water_full):
    _, B, g = water_full
    rng = np.random.default_rng(7)
    D = rng.standard_normal((B.nbf, B.nbf))
    D = D + D.T
    J, K, nq = B.jk(D)
    assert nq == 1035
    assert np.abs(J - np.einsum("pqrs,rs->pq", g, D)).max() < 1e-12
    assert np.abs(K - np.einsum("prqs,rs->pq", g, D)).max() < 1e-12


def test_jk_rank_one_trace_identity(water_full):
    # D = 2 c c^T:  Tr(D J) = Tr(D K)
    _, B, _ = water_full
    c = np.random.default_rng(2).standard_normal(B.nbf)
    D = 2 * np.outer(c, c)
    J, K, _ = B.jk(D)
    assert np.sum(D * J) == pytest.approx(np.sum(D * K), rel=1e-12)


def test_screening_drops_only_small_quartets():
    m = workload("water")
    B = OracleBasis(m)
    D = np.random.default_rng(4).standard_normal((B.nbf, B.nbf))
    D = D + D.T
    J0, K0, n0 = B.jk(D)
    J1, K1, n1 = B.jk(D, tau=1e-3)
    assert n1 < n0
    Q = B.schwarz()
    # error bounded by the skipped products times |D| (Schwarz inequality)
    bound = 1e-3 * np.abs(D).sum() * 8
    assert np.abs(J1 - J0).max() <= bound and np.abs(K1 - K0).max() <= bound


# ---------------------------------------------------------------- linear algebra + SCF (Sec. 3.2)
def test_jacobi_matches_lapack():
    A = np.random.default_rng(9).standard_normal((30, 30))
    A = A + A.T
    w, V = jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
    assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-11)
    assert np.allclose(V.T @ V, np.eye(30), atol=1e-12)


def test_two_centre_closed_form_energy():
    # symmetric two-centre, one s function each: the occupied MO is fixed by symmetry,
    # sigma = (phi1 + phi2)/sqrt(2(1+S)); E follows from s-type closed forms
    a, R = 0.6, 1.4
    m = make_mol([(1, (0, 0, 0)), (1, (0, 0, R))], [(0, 0, (a,), (1.0,)), (1, 0, (a,), (1.0,))])
    B = OracleBasis(m)
    N = (2 * a / math.pi) ** 0.75
    p = 2 * a
    S12 = N * N * (math.pi / p) ** 1.5 * math.exp(-a / 2 * R * R)
    T11 = N * N * (a / 2) * 3 * (math.pi / p) ** 1.5
    T12 = N * N * (a / 2) * (3 - a * R * R) * (math.pi / p) ** 1.5 * math.exp(-a / 2 * R * R)
    f0 = lambda T: 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    V11 = -N * N * 2 * math.pi / p * (f0(0) + f0(p * R * R))
    V12 = -N * N * 2 * math.pi / p * math.exp(-a / 2 * R * R) * 2 * f0(p * (R / 2) ** 2)
    h11, h12 = T11 + V11, T12 + V12

    def ss(c, al):  # (ss|ss) of four single-primitive s functions, closed form
        P = (al[0] * c[0] + al[1] * c[1]) / (al[0] + al[1])
        Q = (al[2] * c[2] + al[3] * c[3]) / (al[2] + al[3])
        pp, qq = al[0] + al[1], al[2] + al[3]
        alpha = pp * qq / (pp + qq)
        kab = math.exp(-al[0] * al[1] / pp * (c[0] - c[1]) ** 2)
        kcd = math.exp(-al[2] * al[3] / qq * (c[2] - c[3]) ** 2)
        return N ** 4 * 2 * math.pi ** 2.5 / (pp * qq * math.sqrt(pp + qq)) * kab * kcd * f0(alpha * (P - Q) ** 2)
    A4 = [a] * 4
    g1111 = ss([0, 0, 0, 0], A4)
    g1122 = ss([0, 0, R, R], A4)
    g1212 = ss([0, R, 0, R], A4)
    g1112 = ss([0, 0, 0, R], A4)
    gggg = (2 * g1111 + 2 * g1122 + 4 * g1212 + 8 * g1112) / (4 * (1 + S12) ** 2)
    hgg = (h11 + h12) / (1 + S12)
    E_ref = 2 * hgg + gggg + 1.0 / R
    S, H = B.onee("S"), B.onee("T") + B.onee("V")
    jk = lambda D: B.jk(D)[:2]
    r = rhf(S, H, jk, 2, B.enuc())
    assert r.converged
    assert r.e_total == pytest.approx(E_ref, abs=1e-11)


@pytest.fixture(scope="module")
def water_scf():
    m = workload("water")
    B = OracleBasis(m)
    S, H = B.onee("S"), B.onee("T") + B.onee("V")
    jk = lambda D: B.jk(D)[:2]
    return m, B, S, H, jk, rhf(S, H, jk, m.nelec, B.enuc())


def test_scf_invariants(water_scf):
    m, B, S, H, jk, r = water_scf
    assert r.converged
    D = r.D
    assert np.trace(D @ S) == pytest.approx(m.nelec, abs=1e-10)
    assert np.abs(D @ S @ D - 2 * D).max() < 1e-8
    J, K = jk(D)
    F = H + J - 0.5 * K
    assert np.abs(F @ D @ S - S @ D @ F).max() < 1e-6


def test_scf_variational(water_scf):
    m, B, S, H, jk, r = water_scf
    # the core guess and random idempotent trial densities all lie above the converged energy
    def energy(D):
        J, K = jk(D)
        return 0.5 * np.sum(D * (2 * H + J - 0.5 * K)) + B.enuc()
    assert r.energies[0] > r.e_total
    X, _ = orthogonaliser(S)
    rng = np.random.default_rng(0)
    for _ in range(4):
        Qm, _ = np.linalg.qr(rng.standard_normal((B.nbf, B.nbf)))
        C = X @ Qm[:, : m.nelec // 2]
        assert energy(2 * C @ C.T) >= r.e_total - 1e-10


def test_scf_diis_off_same_energy(water_scf):
    m, B, S, H, jk, r = water_scf
    r2 = rhf(S, H, jk, m.nelec, B.enuc(), diis=False, max_iter=400)
    assert r2.converged and r2.iters > r.iters
    assert r2.e_total == pytest.approx(r.e_total, abs=1e-9)


def test_scf_rotation_invariance(water_scf):
    m, B, S, H, jk, r = water_scf
    th = 1.1
    Rm = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    m2 = make_mol([(z, tuple(Rm @ x + np.array([0.5, -1.0, 2.0]))) for z, x in zip(m.Z, m.xyz)],
                  [(s.atom, s.l, s.alpha, s.coef) for s in m.shells])
    B2 = OracleBasis(m2)
    S2, H2 = B2.onee("S"), B2.onee("T") + B2.onee("V")
    r2 = rhf(S2, H2, lambda D: B2.jk(D)[:2], m.nelec, B2.enuc())
    assert r2.e_total == pytest.approx(r.e_total, abs=1e-9)


# ---------------------------------------------------------------- spherical (real solid-harmonic) basis
def _sph_scf(mol):
    from oracle import SphericalOracleBasis
    B = SphericalOracleBasis(mol)
    S, H = B.onee("S"), B.onee("T") + B.onee("V")
    return B, rhf(S, H, lambda D: B.jk(D)[:2], mol.nelec, B.enuc())


def test_spherical_d_shell_orthonormal_and_free_of_r2():
    # the five d functions of a shell are orthonormal (only their norms are imposed),
    # and none overlaps an s shell on the same atom, while Cartesian xx does
    from fsim_synth import water_cluster
    from oracle import SphericalOracleBasis
    mol = water_cluster(1, geom_seed=3)
    B = SphericalOracleBasis(mol)
    assert B.nbf == B.nbf_cart - sum(1 for s in mol.shells if s.l == 2)
    S = B.onee("S")
    Sc = B.cart.onee("S")
    off = 0
    for s in mol.shells:
        n = 2 * s.l + 1
        if s.l == 2:
            assert np.abs(S[off:off + n, off:off + n] - np.eye(5)).max() < 1e-13
            d_rows = range(off, off + n)
            for t, u in enumerate(mol.shells):
                if u.l == 0 and u.atom == s.atom:
                    o = sum(2 * v.l + 1 for v in mol.shells[:t])
                    assert max(abs(S[o, r]) for r in d_rows) < 1e-13
                    oc = int(B.cart.ao[t])
                    assert abs(Sc[oc, int(B.cart.ao[mol.shells.index(s)])]) > 0.05  # <s|xx> != 0
        off += n


def test_spherical_f_shell_orthonormal_and_free_of_r2_p():
    # the seven f functions of a shell are orthonormal (only their norms are imposed)
    # and none overlaps a p shell on the same atom; the Cartesian f shell holds
    # r^2 x, r^2 y, r^2 z, which do overlap it (x^3 and xyy here)
    from oracle import SphericalOracleBasis
    mol = make_mol([(8, (0.0, 0.0, 0.0)), (1, (0.0, 1.1, 1.4))],
                   [(0, 0, (0.3, 1.2), (0.6, 0.5)), (0, 1, (0.4, 1.5), (0.5, 0.7)),
                    (0, 3, (0.5, 1.4), (0.8, 0.3)), (1, 0, (0.5,), (1.0,))])
    B = SphericalOracleBasis(mol)
    assert B.nbf == B.nbf_cart - 3
    S, Sc = B.onee("S"), B.cart.onee("S")
    fs, ps = 1 + 3, 1  # spherical offsets: s, p, f, s
    assert np.abs(S[fs:fs + 7, fs:fs + 7] - np.eye(7)).max() < 1e-13
    assert np.abs(S[ps:ps + 3, fs:fs + 7]).max() < 1e-13
    fc = int(B.cart.ao[2])
    assert abs(Sc[ps, fc + 0]) > 0.05 and abs(Sc[ps, fc + 3]) > 0.01  # <x|xxx>, <x|xyy>


def test_spherical_equals_cartesian_without_d():
    from oracle import OracleBasis, SphericalOracleBasis
    from fsim_synth import workload
    mol = workload("water")
    Bs, Bc = SphericalOracleBasis(mol), OracleBasis(mol)
    assert Bs.nbf == Bc.nbf
    for w in "STV":
        assert np.abs(Bs.onee(w) - Bc.onee(w)).max() < 1e-14


def test_spherical_energy_variational_and_rotation_invariant():
    # the spherical space is a subspace of the Cartesian one (E_sph >= E_cart), and a
    # rotation-invariant one: the energy of the rotated molecule is unchanged (a wrong
    # d combination would span a subspace that rotates differently)
    from fsim_synth import water_cluster
    from oracle import OracleBasis
    mol = water_cluster(1, geom_seed=3)
    Bc = OracleBasis(mol)
    Sc, Hc = Bc.onee("S"), Bc.onee("T") + Bc.onee("V")
    rc = rhf(Sc, Hc, lambda D: Bc.jk(D)[:2], mol.nelec, Bc.enuc())
    _, rs = _sph_scf(mol)
    assert rs.converged and rc.converged
    assert rs.e_total > rc.e_total + 1e-6
    th = 0.7
    Rm = np.array([[1.0, 0, 0], [0, math.cos(th), -math.sin(th)], [0, math.sin(th), math.cos(th)]])
    Rm = Rm @ np.array([[math.cos(1.9), 0, math.sin(1.9)], [0, 1.0, 0], [-math.sin(1.9), 0, math.cos(1.9)]])
    m2 = make_mol([(z, tuple(Rm @ x)) for z, x in zip(mol.Z, mol.xyz)],
                  [(s.atom, s.l, s.alpha, s.coef) for s in mol.shells])
    _, rs2 = _sph_scf(m2)
    assert rs2.e_total == pytest.approx(rs.e_total, abs=1e-9)


# ---------------------------------------------------------------- learned-guess network (FP64 reference)
def test_mlp_oracle_gradient_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    nin, w, nout, b = 5, 7, 4, 6
    p = rng.standard_normal(mlp.nparams(nin, w, nout)) * 0.5
    x = rng.standard_normal((b, nin))
    t = rng.standard_normal((b, nout))
    mask = (rng.random((b, nout)) > 0.3).astype(float)
    g = mlp.grad(p, x, t, mask, nin, w, nout)
    h = 1e-6
    for i in rng.choice(len(p), 25, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, t, mask, nin, w, nout) - mlp.loss(p - e, x, t, mask, nin, w, nout)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
