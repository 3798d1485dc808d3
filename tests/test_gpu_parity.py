"""Parity of the CUDA path (through the C-ABI) against the CPU oracle.

Tolerances (FP64 path): ERIs 1e-10 max-abs; J, K 1e-10 max-abs (each element
is a sum of <= nbf^2 products of O(1) magnitude, so FP64 round-off in a
different summation order stays far below); total energy 1e-8 Eh.
Mixed path: J, K within 2e-6 relative to max|J| (FP32 integrals, ~1e-7
relative per integral, accumulated in FP64); with FP64 resets the SCF energy
within 1e-8 Eh of the oracle.
"""
import numpy as np
import pytest

from fsim_synth import workload

from .helpers import make_mol, random_mol

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


# ------------------------------------------------------------------ one-electron
@pytest.mark.parametrize("name", ["water", "water2"])
def test_onee_matches_oracle(name):
    gb, ob = _pair(workload(name))
    for w in "STV":
        assert np.abs(gb.onee(w) - ob.onee(w)).max() < 1e-11, w
    assert gb.enuc() == pytest.approx(ob.enuc(), abs=1e-12)


# ------------------------------------------------------------------ ERIs
def test_eri_dump_water():
    gb, ob = _pair(workload("water"))
    g = gb.eri_dump()
    assert np.abs(g - ob.eri_full()).max() < 1e-10


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eri_dump_random_spd(seed):
    # every class pair up to (dd|dd), 1-3 primitives, random centres
    mol = random_mol(np.random.default_rng(100 + seed), natom=2, lmax=2, nprim=1 + seed)
    gb, ob = _pair(mol)
    assert gb.nbf <= 64
    g = gb.eri_dump()
    ref = ob.eri_full()
    assert np.abs(g - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())


def test_schwarz_matches_oracle():
    gb, ob = _pair(workload("water2"))
    assert np.abs(gb.schwarz() - ob.schwarz()).max() < 1e-12


def test_eri_blocks_sampled_full_size_cluster():
    # (H2O)_8 at full size: sampled quartets of every class, one by one on both sides
    mol = workload("water8")
    gb, ob = _pair(mol)
    ls = [s.l for s in mol.shells]
    rng = np.random.default_rng(5)
    by_l = {l: [i for i, x in enumerate(ls) if x == l] for l in (0, 1, 2)}
    quartets = []
    for combo in [(2, 2, 2, 2), (2, 1, 2, 0), (1, 1, 1, 1), (0, 0, 0, 0), (2, 2, 1, 0), (0, 2, 1, 2),
                  (1, 0, 2, 2), (2, 0, 0, 2)]:
        for _ in range(3):
            quartets.append([int(rng.choice(by_l[l])) for l in combo])
    blocks = gb.eri_quartets(quartets)
    for q, blk in zip(quartets, blocks):
        ref = ob.eri_block(*q)
        assert np.abs(blk - ref).max() < 1e-10, q



def test_eri_blocks_sampled_organic_cloud():
    # organic cloud of 60 heavy atoms (1140 Cartesian functions): a seeded sample of
    # 10^5 shell quartets drawn uniformly, plus 8 quartets of every (la lb|lc ld)
    # combination drawn among shells of neighbouring atoms, FP64 blocks one by one
    mol = workload("cloud60")
    gb, ob = _pair(mol)
    ls = np.array([s.l for s in mol.shells])
    rng = np.random.default_rng(21)
    quartets = rng.integers(0, mol.nshell, size=(100000, 4))
    xyz = np.asarray(mol.xyz)[[s.atom for s in mol.shells]]
    extra = []
    for combo in np.ndindex(3, 3, 3, 3):
        for _ in range(8):
            a = int(rng.choice(np.flatnonzero(ls == combo[0])))
            near = np.linalg.norm(xyz - xyz[a], axis=1) < 6.0
            extra.append([a] + [int(rng.choice(np.flatnonzero((ls == l) & near))) for l in combo[1:]])
    quartets = np.concatenate([quartets, np.array(extra)]).astype(np.int32)
    got = gb.eri_quartets(quartets)
    ref = ob.eri_blocks(quartets)
    err = max(float(np.abs(g - r).max()) for g, r in zip(got, ref))
    assert err < 1e-10, err


# ------------------------------------------------------------------ J / K
@pytest.mark.parametrize("tau", [0.0, 1e-10, 1e-4])
def test_jk_fp64_water(tau):
    from paper_2510_24968_gb300 import FSIM_FP64
    gb, ob = _pair(workload("water"))
    D = _rand_sym(gb.nbf, 1)
    J, K = gb.fock_build(D, tau=tau, precision=FSIM_FP64)
    Jo, Ko, nq = ob.jk(D, tau=tau)
    assert gb.last_quartet_count() == nq
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10


@pytest.mark.parametrize("seed", [0, 1])
def test_jk_fp64_random_spd(seed):
    from paper_2510_24968_gb300 import FSIM_FP64
    mol = random_mol(np.random.default_rng(200 + seed), natom=3, lmax=2, nprim=2)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, seed)
    J, K = gb.fock_build(D, tau=0.0, precision=FSIM_FP64)
    Jo, Ko, _ = ob.jk(D)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10


def test_jk_mixed_random_spd():
    # FP32 integrals (~1e-7 relative each) accumulated in FP64: 2e-6 of max|J|
    from paper_2510_24968_gb300 import FSIM_MIXED
    mol = random_mol(np.random.default_rng(300), natom=3, lmax=2, nprim=3)
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 3)
    J, K = gb.fock_build(D, tau=0.0, precision=FSIM_MIXED)
    Jo, Ko, _ = ob.jk(D)
    assert np.abs(J - Jo).max() < 2e-6 * np.abs(Jo).max()
    assert np.abs(K - Ko).max() < 2e-6 * np.abs(Jo).max()


def test_jk_mixed_boys_fp64_policy():
    # the optional FP64 Boys branch above T = 30 gives the same J/K within FP32 tolerance
    from paper_2510_24968_gb300 import FSIM_MIXED, FsimError
    mol = workload("water2")
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 6) * 0.1
    Jo, Ko, _ = ob.jk(D, tau=1e-10)
    for t64 in (0.0, 30.0):
        J, K = gb.fock_build(D, tau=1e-10, precision=FSIM_MIXED, boys_fp64_T=t64)
        scale = np.abs(Jo).max()
        assert np.abs(J - Jo).max() < 2e-6 * scale and np.abs(K - Ko).max() < 2e-6 * scale
    with pytest.raises(FsimError):
        gb.fock_build(D, precision=FSIM_MIXED, boys_fp64_T=10.0)


def test_jk_device_pointers_and_shards():
    from paper_2510_24968_gb300 import FSIM_FP64
    gb, ob = _pair(workload("water2"))
    D = _rand_sym(gb.nbf, 4)
    Dt = torch.from_numpy(D).cuda()
    J, K = gb.fock_build(Dt, tau=1e-10, precision=FSIM_FP64)
    torch.cuda.synchronize()
    Js, Ks = torch.zeros_like(Dt), torch.zeros_like(Dt)
    for s in range(3):
        a, b = gb.fock_build(Dt, tau=1e-10, precision=FSIM_FP64, shard=s, nshards=3)
        Js += a
        Ks += b
    torch.cuda.synchronize()
    assert torch.abs(Js - J).max().item() < 1e-11 and torch.abs(Ks - K).max().item() < 1e-11
    Jo, Ko, _ = ob.jk(D, tau=1e-10)
    assert np.abs(J.cpu().numpy() - Jo).max() < 1e-10


def test_jk_sampled_blocks_full_size_cluster():
    # (H2O)_8, tau 1e-10, FP64 and mixed: sampled J/K blocks by definition on the oracle side
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    mol = workload("water8")
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 8) * 0.1
    Q = ob.schwarz()
    J, K = gb.fock_build(D, tau=1e-10, precision=FSIM_FP64)
    Jm, Km = gb.fock_build(D, tau=1e-10, precision=FSIM_MIXED)
    ls = [s.l for s in mol.shells]
    ao = np.cumsum([0] + [(l + 1) * (l + 2) // 2 for l in ls])
    d_shells = [i for i, l in enumerate(ls) if l == 2]
    p_shells = [i for i, l in enumerate(ls) if l == 1]
    s_shells = [i for i, l in enumerate(ls) if l == 0]
    for sa, sb in [(d_shells[0], d_shells[3]), (p_shells[2], s_shells[7]), (s_shells[1], s_shells[30]),
                   (d_shells[5], p_shells[9])]:
        Jb, Kb = ob.jk_block(D, sa, sb, tau=1e-10, Q=Q)
        sl = (slice(ao[sa], ao[sa + 1]), slice(ao[sb], ao[sb + 1]))
        assert np.abs(J[sl] - Jb).max() < 1e-10 and np.abs(K[sl] - Kb).max() < 1e-10
        scale = np.abs(J).max()
        assert np.abs(Jm[sl] - Jb).max() < 2e-6 * scale and np.abs(Km[sl] - Kb).max() < 2e-6 * scale


def test_jk_edge_cases():
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    # single s shell; a screening threshold that removes everything; 4-primitive shells
    m1 = make_mol([(1, (0.0, 0.0, 0.0))], [(0, 0, (0.5,), (1.0,))])
    gb, ob = _pair(m1)
    D = np.array([[0.7]])
    J, K = gb.fock_build(D, tau=0.0)
    Jo, Ko, _ = ob.jk(D)
    assert abs(J[0, 0] - Jo[0, 0]) < 1e-13 and abs(K[0, 0] - Ko[0, 0]) < 1e-13
    J, K = gb.fock_build(D, tau=1e6, precision=FSIM_MIXED)
    assert np.all(J == 0) and np.all(K == 0) and gb.last_quartet_count() == 0
    m4 = make_mol([(8, (0.0, 0.0, 0.0)), (1, (0.0, 1.2, 0.8))],
                  [(0, 2, (0.3, 0.8, 2.0, 5.0), (0.2, 0.5, 0.4, 0.1)), (1, 1, (0.4, 1.3, 3.1, 7.7), (0.3, 0.3, 0.6, 0.2)),
                   (1, 0, (0.25,), (1.0,))])
    gb, ob = _pair(m4)
    D = _rand_sym(gb.nbf, 9)
    J, K = gb.fock_build(D, tau=0.0, precision=FSIM_FP64)
    Jo, Ko, _ = ob.jk(D)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10


def test_invalid_arguments_raise():
    from paper_2510_24968_gb300 import Basis, FsimError
    bad = make_mol([(1, (0.0, 0.0, 0.0))], [(0, 4, (0.5,), (1.0,))])  # g shells are not supported
    with pytest.raises(FsimError):
        Basis(bad)
    gb = Basis(workload("water"))
    with pytest.raises(FsimError):
        gb.fock_build(np.zeros((gb.nbf, gb.nbf)), precision=7)


# ------------------------------------------------------------------ SCF
@pytest.fixture(scope="module")
def water_oracle_scf():
    from oracle import OracleBasis, rhf
    mol = workload("water")
    ob = OracleBasis(mol)
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    return mol, rhf(S, H, lambda D: ob.jk(D)[:2], mol.nelec, ob.enuc())


def test_scf_fp64_water(water_oracle_scf):
    from paper_2510_24968_gb300 import FSIM_FP64, Basis
    mol, ro = water_oracle_scf
    r = Basis(mol).scf(precision=FSIM_FP64, tau=0.0, want_density=True)
    assert r["converged"]
    assert abs(r["e_total"] - ro.e_total) < 1e-8
    assert np.abs(r["D"] - ro.D).max() < 1e-6


@pytest.mark.parametrize("diis", [True, False])
def test_scf_trajectory_water(diis):
    # the SCF iteration itself (Sec. 3.2; DIIS per Algorithm 1, or plain), energy by
    # energy against the oracle's: same guess, same extrapolation, same aufbau
    from oracle import OracleBasis, rhf
    from paper_2510_24968_gb300 import FSIM_FP64, Basis
    mol = workload("water")
    ob = OracleBasis(mol)
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    ro = rhf(S, H, lambda D: ob.jk(D)[:2], mol.nelec, ob.enuc(), max_iter=40, diis=diis)
    r = Basis(mol).scf(precision=FSIM_FP64, tau=0.0, max_iter=40, diis_size=8 if diis else 0)
    n = min(len(ro.energies), len(r["energies"]))
    assert n >= 8 and r["iters"] == ro.iters and r["converged"] == ro.converged
    assert np.abs(np.array(ro.energies[:n]) - r["energies"][:n]).max() < 1e-9


# ------------------------------------------------------------------ spherical basis
def test_spherical_onee_jk_match_oracle():
    # (H2O)_2 with O d shells in the real solid-harmonic basis: S, T, V and J, K of a
    # spherical density against the oracle's own spherical transform
    from oracle import SphericalOracleBasis
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED, Basis
    mol = workload("water2")
    gb, ob = Basis(mol, spherical=True), SphericalOracleBasis(mol)
    assert gb.nbf == ob.nbf and gb.nbf_cart == ob.nbf_cart and gb.nbf < gb.nbf_cart
    for w in "STV":
        assert np.abs(gb.onee(w) - ob.onee(w)).max() < 1e-11, w
    D = _rand_sym(gb.nbf, 14) * 0.1
    Jo, Ko, _ = ob.jk(D, tau=1e-10)
    J, K = gb.fock_build(D, tau=1e-10, precision=FSIM_FP64)
    assert np.abs(J - Jo).max() < 1e-10 and np.abs(K - Ko).max() < 1e-10
    Jm, Km = gb.fock_build(D, tau=1e-10, precision=FSIM_MIXED)
    s = np.abs(Jo).max()
    assert np.abs(Jm - Jo).max() < 2e-6 * s and np.abs(Km - Ko).max() < 2e-6 * s


def test_spherical_scf_energy_matches_oracle():
    from oracle import SphericalOracleBasis, rhf
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED, Basis
    mol = workload("water2")
    ob = SphericalOracleBasis(mol)
    S, H = ob.onee("S"), ob.onee("T") + ob.onee("V")
    ro = rhf(S, H, lambda D: ob.jk(D, tau=1e-10)[:2], mol.nelec, ob.enuc())
    gb = Basis(mol, spherical=True)
    for prec in (FSIM_FP64, FSIM_MIXED):
        r = gb.scf(precision=prec, tau=1e-10)
        assert r["converged"] and abs(r["e_total"] - ro.e_total) < 1e-8, prec
    # the Cartesian energy of the same molecule lies below (larger variational space)
    rc = Basis(mol).scf(precision=FSIM_FP64, tau=1e-10)
    assert rc["e_total"] < ro.e_total - 1e-6


def test_spherical_rejected_where_cartesian_only():
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis, FsimError, scf_batched
    from paper_2510_24968_gb300 import guess
    gb = Basis(workload("water"), spherical=True)
    with pytest.raises(FsimError):
        scf_batched([gb], precision=FSIM_MIXED, tau=1e-10, max_iter=2)
    with pytest.raises(FsimError):
        guess.features(gb)


def test_scf_mixed_water(water_oracle_scf):
    # mixed builds with FP64 resets reach the FP64 energy; without the resets the
    # FP32 error of this near-linearly-dependent basis stays at the 1e-4 Eh level
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis
    mol, ro = water_oracle_scf
    r = Basis(mol).scf(precision=FSIM_MIXED, tau=0.0, final_fp64=True)
    assert r["converged"] and 1 <= r["fp64_builds"] <= 6 and r["mixed_builds"] > r["fp64_builds"]
    assert abs(r["e_total"] - ro.e_total) < 1e-8


def test_scf_full_size_cluster_energy():
    # (H2O)_8 at full size, tau 1e-10: FP64 and mixed (with FP64 resets) within
    # 1e-8 Eh of the oracle's energy written by tests/golden/make_water8_energy.py
    import json
    import os
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED, Basis
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "water8_scf_oracle.json")))
    gb = Basis(workload("water8"))
    r64 = gb.scf(precision=FSIM_FP64, tau=1e-10)
    assert r64["converged"] and abs(r64["e_total"] - gold["e_total"]) < 1e-8
    rmx = gb.scf(precision=FSIM_MIXED, tau=1e-10)
    assert rmx["converged"] and abs(rmx["e_total"] - gold["e_total"]) < 1e-8
    assert rmx["time_s"] < r64["time_s"]


def test_jk_sampled_blocks_organic_cloud():
    # organic cloud of 12 heavy atoms, tau 1e-11: sampled J/K blocks by definition;
    # FP64 within 1e-10, mixed (FP32 Boys everywhere, or FP64 Boys above T = 30)
    # within 2e-6 of max|J|
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED
    mol = workload("cloud12")
    gb, ob = _pair(mol)
    D = _rand_sym(gb.nbf, 12) * 0.05
    Q = ob.schwarz()
    J, K = gb.fock_build(D, tau=1e-11, precision=FSIM_FP64)
    mixed = [gb.fock_build(D, tau=1e-11, precision=FSIM_MIXED, boys_fp64_T=t) for t in (0.0, 30.0)]
    ls = [s.l for s in mol.shells]
    ao = np.cumsum([0] + [(l + 1) * (l + 2) // 2 for l in ls])
    d_shells = [i for i, l in enumerate(ls) if l == 2]
    p_shells = [i for i, l in enumerate(ls) if l == 1]
    s_shells = [i for i, l in enumerate(ls) if l == 0]
    scale = np.abs(J).max()
    for sa, sb in [(d_shells[2], d_shells[7]), (p_shells[5], d_shells[0]), (s_shells[3], s_shells[20])]:
        Jb, Kb = ob.jk_block(D, sa, sb, tau=1e-11, Q=Q)
        sl = (slice(ao[sa], ao[sa + 1]), slice(ao[sb], ao[sb + 1]))
        assert np.abs(J[sl] - Jb).max() < 1e-10 and np.abs(K[sl] - Kb).max() < 1e-10
        for Jm, Km in mixed:
            assert np.abs(Jm[sl] - Jb).max() < 2e-6 * scale and np.abs(Km[sl] - Kb).max() < 2e-6 * scale
