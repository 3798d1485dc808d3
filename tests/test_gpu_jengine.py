"""Coulomb-only builds by the Hermite-space J-engine (fsim_j_build) through the C-ABI.

J_mu,nu = sum D_la,si (mu nu|la si) (Eq. fock) against the oracle's J element
by element: 1e-10 max-abs in FP64 and 2e-6 of max|J| in mixed precision, the
tolerances of the fused J/K build; against the fused build's J on the full
(H2O)_8 cluster and the 12-atom organic cloud (same screened quartet set, both
orders); shard sums; the ordered quartet count; rejected options.
"""
import numpy as np
import pytest

from fsim_synth import workload

from .helpers import random_mol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_24968_gb300.build import build
    build()
    yield


def _pair(mol):
    from oracle import OracleBasis
    from paper_2510_24968_gb300 import Basis
    return Basis(mol), OracleBasis(mol)


def _rand_sym(n, seed):
    D = np.random.default_rng(seed).standard_normal((n, n))
    return D + D.T


def test_j_engine_water_against_oracle():
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    gb, ob = _pair(workload("water"))
    D = _rand_sym(gb.nbf, 3)
    Jo, _, nq = ob.jk(D)
    J = gb.j_build(D, tau=0.0, precision=FSIM_FP64)
    assert np.abs(J - Jo).max() < 1e-10
    # every ordered pair of the 45 shell pairs
    assert gb.last_quartet_count() == 45 * 45 == 2 * nq - 45
    Jm = gb.j_build(D, tau=0.0, precision=FSIM_MIXED)
    assert np.abs(Jm - Jo).max() < 2e-6 * np.abs(Jo).max()


@pytest.mark.parametrize("seed,nprim", [(0, 2), (1, 3), (2, 1)])
def test_j_engine_random_spd_against_oracle(seed, nprim):
    # every class pair up to (dd|dd) in both orders; T past the Boys table
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    mol = random_mol(np.random.default_rng(500 + seed), natom=3, lmax=2, nprim=nprim)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 50 + seed)
    Jo, _, _ = ob.jk(D)
    J = gb.j_build(D, tau=0.0, precision=FSIM_FP64)
    assert np.abs(J - Jo).max() < 1e-10
    for b64 in (0.0, 30.0):
        Jm = gb.j_build(D, tau=0.0, precision=FSIM_MIXED, boys_fp64_T=b64)
        assert np.abs(Jm - Jo).max() < 2e-6 * np.abs(Jo).max()


@pytest.mark.parametrize("name,tau", [("water8", 1e-10), ("cloud12", 1e-11)])
def test_j_engine_equals_fused_build(name, tau):
    # the same screened quartets in both orders: J equals the fused J/K build's J,
    # with device pointers, and sampled blocks match the oracle's by-definition sums
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    mol = workload(name)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 7) * 0.05
    Dt = torch.from_numpy(D).cuda()
    for prec, tol in ((FSIM_FP64, 1e-10), (FSIM_MIXED, None)):
        Jf, _ = gb.fock_build(Dt, tau=tau, precision=prec)
        nq_fused = gb.last_quartet_count()
        J = gb.j_build(Dt, tau=tau, precision=prec)
        torch.cuda.synchronize()
        assert nq_fused < gb.last_quartet_count() <= 2 * nq_fused
        err = torch.abs(J - Jf).max().item()
        assert err < (tol if tol else 2e-6 * torch.abs(Jf).max().item()), (prec, err)
    J = J.cpu().numpy()
    Q = ob.schwarz()
    ls = [s.l for s in mol.shells]
    ao = np.cumsum([0] + [(l + 1) * (l + 2) // 2 for l in ls])
    d_shells = [i for i, l in enumerate(ls) if l == 2]
    s_shells = [i for i, l in enumerate(ls) if l == 0]
    Jfp = gb.j_build(D, tau=tau, precision=FSIM_FP64)
    for sa, sb in [(d_shells[0], d_shells[1]), (s_shells[2], d_shells[0])]:
        Jb, _ = ob.jk_block(D, sa, sb, tau=tau, Q=Q)
        sl = (slice(ao[sa], ao[sa + 1]), slice(ao[sb], ao[sb + 1]))
        assert np.abs(Jfp[sl] - Jb).max() < 1e-10


def test_j_engine_shards_sum_to_the_whole():
    from paper_2510_24968_gb300 import FSIM_FP64
    gb, _ = _pair(workload("water4"))
    D = _rand_sym(gb.nbf, 9) * 0.1
    J = gb.j_build(D, tau=1e-10, precision=FSIM_FP64)
    Js = sum(gb.j_build(D, tau=1e-10, precision=FSIM_FP64, shard=k, nshards=3) for k in range(3))
    assert np.abs(Js - J).max() < 1e-11


def test_j_engine_rejects_unsupported_options():
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_FP64, Basis, FsimError
    mol = workload("water")
    gb = Basis(mol)
    D = _rand_sym(gb.nbf, 1)
    with pytest.raises(FsimError):
        gb.j_build(D, precision=FSIM_DFLOAT)
    with pytest.raises(FsimError):
        gb.j_build(D, precision=FSIM_FP64, boys_fp64_T=10.0)
    sph = Basis(mol, spherical=True)
    with pytest.raises(FsimError):
        sph.j_build(np.zeros((sph.nbf, sph.nbf)))
