"""Double-float Fock builds (FSIM_DFLOAT) against the CPU oracle, through the C-ABI.

Tolerances are the FP64 path's: J, K 1e-10 max-abs, energies 1e-8 Eh.  A
double-float value carries about 48 significant bits (relative rounding
2^-47 per operation, 64 times FP64's); an integral of O(1) magnitude that
passes through a few hundred such operations keeps its error near 1e-13, and
J, K sum at most nbf^2 of them, so the FP64 bar leaves about two orders of
margin.  By default a double-float build runs the double-float kernel for
class pairs of total angular momentum <= 4 and the FP64 kernel for the rest;
test_jk_every_kernel_and_shape forces every double-float kernel (all but
(dd|dp) and (dd|dd), which have none) through fsim_set_launch.
"""
import json
import os

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


@pytest.mark.parametrize("tau", [0.0, 1e-10])
def test_jk_dfloat_water(tau):
    from paper_2510_24968_gb300 import FSIM_DFLOAT
    gb, ob = _pair(workload("water"))
    D = _rand_sym(gb.nbf, 21)
    J, K = gb.fock_build(D, tau=tau, precision=FSIM_DFLOAT)
    Jo, Ko, nq = ob.jk(D, tau=tau)
    assert gb.last_quartet_count() == nq
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_jk_dfloat_random_spd(seed):
    # every class pair up to (dd|dd); T from 0 to beyond the Boys table (asymptotic branch)
    from paper_2510_24968_gb300 import FSIM_DFLOAT
    mol = random_mol(np.random.default_rng(400 + seed), natom=3, lmax=2, nprim=2)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 30 + seed)
    J, K = gb.fock_build(D, tau=0.0, precision=FSIM_DFLOAT)
    Jo, Ko, _ = ob.jk(D)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10


def test_jk_dfloat_device_pointers_and_autotune():
    # device pointers; the autotuned launch shapes give the same J, K up to rounding order
    from paper_2510_24968_gb300 import FSIM_DFLOAT
    gb, ob = _pair(workload("water2"))
    D = _rand_sym(gb.nbf, 22)
    Dt = torch.from_numpy(D).cuda()
    J, K = gb.fock_build(Dt, tau=1e-10, precision=FSIM_DFLOAT)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    Jo, Ko, _ = ob.jk(D, tau=1e-10)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10
    choice = gb.autotune(tau=1e-10, precision=FSIM_DFLOAT)
    assert choice and all(v[0] > 0 for v in choice.values())  # no cooperative kernel in double-float
    Jt, Kt = gb.fock_build(Dt, tau=1e-10, precision=FSIM_DFLOAT)
    assert np.abs(Jt.cpu().numpy() - Jo).max() < 1e-10 and np.abs(Kt.cpu().numpy() - Ko).max() < 1e-10


@pytest.mark.parametrize("prec_name", ["fp64", "mixed", "dfloat"])
def test_jk_every_kernel_and_shape(prec_name):
    # every kernel of a precision, forced through fsim_set_launch on every class pair
    # up to (dd|dd): one and three threads per quartet's bra primitive pairs, the
    # cooperative kernel (FP64, mixed), and in double-float builds both the
    # double-float and the FP64 kernel
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_FP64, FSIM_MIXED, FsimError
    prec = {"fp64": FSIM_FP64, "mixed": FSIM_MIXED, "dfloat": FSIM_DFLOAT}[prec_name]
    mol = random_mol(np.random.default_rng(410), natom=3, lmax=2, nprim=2)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 41)
    Jo, Ko, _ = ob.jk(D)
    tol = (lambda M: 2e-6 * np.abs(Jo).max()) if prec == FSIM_MIXED else (lambda M: 1e-10)
    pairs = [(x, y) for x in range(6) for y in range(x + 1)]
    variants = [11, 31] + ([1011, 1031] if prec == FSIM_DFLOAT else [-1])
    for v in variants:
        ch = {}
        for (x, y) in pairs:
            ch[(x, y)] = v if not (prec == FSIM_DFLOAT and x == 5 and y >= 4 and v < 1000) else v + 1000
        gb.set_launch(ch, tau=0.0, precision=prec)
        J, K = gb.fock_build(D, tau=0.0, precision=prec)
        assert np.abs(J - Jo).max() < tol(J) and np.abs(K - Ko).max() < tol(K), v
    with pytest.raises(FsimError):
        gb.set_launch({(0, 0): 91}, tau=0.0, precision=prec)  # 9 threads > 4 primitive pairs
    with pytest.raises(FsimError):
        gb.set_launch({(5, 5): 271}, tau=0.0, precision=prec)  # 27 threads need 9 bra primitive pairs
    if prec == FSIM_DFLOAT:
        with pytest.raises(FsimError):
            gb.set_launch({(5, 5): 11}, tau=0.0, precision=prec)  # no double-float (dd|dd) kernel


@pytest.mark.parametrize("name,tau", [("water8", 1e-10), ("cloud12", 1e-11)])
def test_jk_dfloat_sampled_blocks(name, tau):
    # full-size (H2O)_8 and the 12-atom organic cloud: sampled J/K blocks by definition
    # on the oracle side, and the whole J/K against the FP64 build
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_FP64
    mol = workload(name)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 23) * 0.05
    Q = ob.schwarz()
    J, K = gb.fock_build(D, tau=tau, precision=FSIM_DFLOAT)
    J64, K64 = gb.fock_build(D, tau=tau, precision=FSIM_FP64)
    assert np.abs(J - J64).max() < 1e-10 and np.abs(K - K64).max() < 1e-10
    ls = [s.l for s in mol.shells]
    ao = np.cumsum([0] + [(l + 1) * (l + 2) // 2 for l in ls])
    d_shells = [i for i, l in enumerate(ls) if l == 2]
    p_shells = [i for i, l in enumerate(ls) if l == 1]
    s_shells = [i for i, l in enumerate(ls) if l == 0]
    for sa, sb in [(d_shells[0], d_shells[3]), (p_shells[2], d_shells[1]), (s_shells[1], s_shells[9])]:
        Jb, Kb = ob.jk_block(D, sa, sb, tau=tau, Q=Q)
        sl = (slice(ao[sa], ao[sa + 1]), slice(ao[sb], ao[sb + 1]))
        assert np.abs(J[sl] - Jb).max() < 1e-10 and np.abs(K[sl] - Kb).max() < 1e-10


def test_scf_dfloat_water():
    # every build in double-float: the oracle's SCF energy
    from oracle import OracleBasis, rhf
    from paper_2510_24968_gb300 import FSIM_DFLOAT, Basis
    mol = workload("water")
    ob = OracleBasis(mol)
    ro = rhf(ob.onee("S"), ob.onee("T") + ob.onee("V"), lambda D: ob.jk(D)[:2], mol.nelec, ob.enuc())
    r = Basis(mol).scf(precision=FSIM_DFLOAT, tau=0.0)
    assert r["converged"] and abs(r["e_total"] - ro.e_total) < 1e-8


def test_scf_mixed_with_dfloat_resets_full_size_cluster():
    # (H2O)_8, tau 1e-10: mixed builds whose resets are double-float builds reach the
    # oracle's energy (tests/golden/make_water8_energy.py) within 1e-8 Eh
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "water8_scf_oracle.json")))
    r = Basis(workload("water8")).scf(precision=FSIM_MIXED, tau=1e-10, final_fp64=2)
    assert r["converged"] and r["fp64_builds"] >= 1
    assert abs(r["e_total"] - gold["e_total"]) < 1e-8


def test_dfloat_bad_options_rejected():
    # an unknown reset mode; the batched paths, which have FP64 and mixed builds only
    from paper_2510_24968_gb300 import FSIM_DFLOAT, FSIM_MIXED, Basis, Batch, FsimError, scf_batched
    gb = Basis(workload("water"))
    with pytest.raises(FsimError):
        gb.scf(precision=FSIM_MIXED, tau=0.0, final_fp64=3)
    with pytest.raises(FsimError):
        scf_batched([gb], precision=FSIM_DFLOAT, tau=1e-10, max_iter=2)
    D = torch.zeros((gb.nbf, gb.nbf), dtype=torch.float64, device="cuda")
    bt = Batch([gb], [D], [torch.zeros_like(D)], [torch.zeros_like(D)], tau=1e-10)
    with pytest.raises(FsimError):
        bt.fock(FSIM_DFLOAT)
    bt.close()
