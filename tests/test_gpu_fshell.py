"""f shells (l = 3) through the C-ABI against the oracle.

Every class pair that holds an f shell runs the runtime-angular-momentum
kernel (csrc/generic.cuh); the s/p/d class pairs of the same molecules keep
the unrolled kernels.  Tolerances are those of the s/p/d tests: one-electron
1e-11, Schwarz 1e-12, ERIs and FP64 (and double-float) J/K 1e-10, mixed J/K
2e-6 of max|J|, SCF energies 1e-8 Eh; spherical f (seven real solid
harmonics) against the oracle's own transform.
"""
import numpy as np
import pytest

from .helpers import make_mol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_24968_gb300.build import build
    build()
    yield


def _water_f():
    # water with an f polarisation shell on O (and a d shell), 2-3 primitives
    O, H1, H2 = (0.0, 0.0, 0.0), (1.4305, 1.1093, 0.0), (-1.4305, 1.1093, 0.0)
    sh = [(0, 0, (0.15, 0.4, 1.1), (0.5, 0.7, 0.3)), (0, 0, (0.6, 1.6, 4.2), (0.4, 0.6, 0.5)),
          (0, 1, (0.25, 0.7, 1.9), (0.6, 0.5, 0.4)), (0, 2, (0.5, 1.3), (0.7, 0.4)),
          (0, 3, (0.6, 1.5), (0.8, 0.3)),
          (1, 0, (0.2, 0.6, 1.7), (0.5, 0.6, 0.3)), (2, 0, (0.2, 0.6, 1.7), (0.5, 0.6, 0.3))]
    return make_mol([(8, O), (1, H1), (1, H2)], sh, "water_f")


def _spdf_pair():
    # two atoms, s, p, d and f shells on each: every f class pair up to (ff|ff)
    rng = np.random.default_rng(31)
    atoms = [(6, (0.0, 0.0, 0.0)), (7, tuple(rng.uniform(-1.5, 1.5, 3)))]
    sh = []
    for a in range(2):
        for l in range(4):
            al = tuple(sorted(rng.uniform(0.3, 2.0, 2)))
            sh.append((a, l, al, tuple(rng.uniform(0.3, 1.0, 2))))
    return make_mol(atoms, sh, "spdf2")


def _pair(mol, spherical=False):
    from oracle import OracleBasis, SphericalOracleBasis
    from paper_2510_24968_gb300 import Basis
    return Basis(mol, spherical=spherical), (SphericalOracleBasis(mol) if spherical else OracleBasis(mol))


def _rand_sym(n, seed):
    D = np.random.default_rng(seed).standard_normal((n, n))
    return D + D.T


@pytest.mark.parametrize("make", [_water_f, _spdf_pair])
def test_f_one_electron_schwarz_and_eris(make):
    mol = make()
    gb, ob = _pair(mol)
    for w in "STV":
        assert np.abs(gb.onee(w) - ob.onee(w)).max() < 1e-11, w
    assert np.abs(gb.schwarz() - ob.schwarz()).max() < 1e-12
    g = gb.eri_dump()
    go = ob.eri_full()
    assert np.abs(g - go).max() < 1e-10


@pytest.mark.parametrize("make", [_water_f, _spdf_pair])
@pytest.mark.parametrize("tau", [0.0, 1e-10])
def test_f_jk_all_precisions(make, tau):
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_FP64, FSIM_MIXED
    mol = make()
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 5)
    Jo, Ko, nq = ob.jk(D, tau=tau)
    J, K = gb.fock_build(D, tau=tau, precision=FSIM_FP64)
    assert gb.last_quartet_count() == nq
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10
    Jd, Kd = gb.fock_build(D, tau=tau, precision=FSIM_DFLOAT)
    assert np.abs(Jd - Jo).max() < 1e-10 and np.abs(Kd - Ko).max() < 1e-10
    Jm, Km = gb.fock_build(D, tau=tau, precision=FSIM_MIXED)
    s = np.abs(Jo).max()
    assert np.abs(Jm - Jo).max() < 2e-6 * s and np.abs(Km - Ko).max() < 2e-6 * s
    # device pointers
    Dt = torch.from_numpy(D).cuda()
    Jt, Kt = gb.fock_build(Dt, tau=tau, precision=FSIM_FP64)
    assert np.abs(Jt.cpu().numpy() - Jo).max() < 1e-10 and np.abs(Kt.cpu().numpy() - Ko).max() < 1e-10


def test_f_scf_energy_against_oracle():
    from oracle import rhf
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    mol = _water_f()
    gb, ob = _pair(mol)
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    ro = rhf(S, H, lambda d: ob.jk(d)[:2], mol.nelec, ob.enuc())
    assert ro.converged
    r64 = gb.scf(precision=FSIM_FP64, tau=0.0)
    rmx = gb.scf(precision=FSIM_MIXED, tau=0.0)
    assert r64["converged"] and abs(r64["e_total"] - ro.e_total) < 1e-8
    assert rmx["converged"] and abs(rmx["e_total"] - ro.e_total) < 1e-8


def test_spherical_f_against_oracle_transform():
    from oracle import rhf
    from paper_2510_24968_gb300 import FSIM_FP64
    mol = _water_f()
    gb, ob = _pair(mol, spherical=True)
    assert gb.nbf == ob.nbf == 19  # s s p d f s s: 1 + 1 + 3 + 5 + 7 + 1 + 1
    for w in "STV":
        assert np.abs(gb.onee(w) - ob.onee(w)).max() < 1e-11, w
    D = _rand_sym(gb.nbf, 8)
    J, K = gb.fock_build(D, tau=0.0, precision=FSIM_FP64)
    Jo, Ko, _ = ob.jk(D)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    ro = rhf(S, H, lambda d: ob.jk(d)[:2], mol.nelec, ob.enuc())
    r = gb.scf(precision=FSIM_FP64, tau=0.0)
    assert r["converged"] and abs(r["e_total"] - ro.e_total) < 1e-8


def test_f_bases_refused_where_unsupported():
    from paper_2510_24968_gb300 import FSIM_FP64, FsimError, scf_batched
    gb, _ = _pair(_water_f())
    D = _rand_sym(gb.nbf, 1)
    with pytest.raises(FsimError):
        gb.j_build(D, precision=FSIM_FP64)
    with pytest.raises(FsimError):
        scf_batched([gb], precision=FSIM_FP64)
