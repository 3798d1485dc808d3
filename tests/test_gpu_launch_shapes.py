"""Parity of every launch shape of the hot J/K kernels, through the C-ABI.

The autotuner may give each class pair any of twelve shapes of the unrolled
kernel -- each quartet's primitive quartets split over psplit = 1, 3, 9 or 27
threads (bra primitive pairs first, 27 splitting the ket primitive pairs as
well), its ket-component chunks shared out over csplit = 1, 2 or 4 warp
groups -- or the warp-cooperative kernel.  Each is forced here through
fsim_set_launch on every class pair up to (dd|dd) of a molecule with
3-primitive s, p and d shells (9 primitive pairs, so psplit = 9 and 27 are
legal), in FP64 and in mixed precision, and J, K are compared element by
element with the oracle's (Eq. fock): 1e-10 max-abs for FP64, 2e-6 of max|J|
for mixed.  A molecule whose shells have 1 to 4 primitives (1 to 16 primitive
pairs per shell pair) runs the split shapes with ragged primitive counts.

The 60-heavy-atom organic cloud (1140 functions) is also built whole in mixed
precision through the hot kernel, with a density that lives on a handful of
neighbouring shells; sampled J/K blocks are checked against the oracle's
by-definition block sums (which skip the zero density blocks).
"""
import itertools

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


PAIRS = [(x, y) for x in range(6) for y in range(x + 1)]


@pytest.fixture(scope="module")
def spd3():
    from oracle import OracleBasis
    from paper_2510_24968_gb300 import Basis
    mol = random_mol(np.random.default_rng(777), natom=3, lmax=2, nprim=3, spread=1.6)
    gb, ob = Basis(mol), OracleBasis(mol)
    D = np.random.default_rng(78).standard_normal((gb.nbf, gb.nbf))
    D = D + D.T
    Jo, Ko, _ = ob.jk(D)
    return gb, D, Jo, Ko


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_every_launch_shape_every_class_pair(spd3, prec_name):
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED, FsimError
    prec = {"fp64": FSIM_FP64, "mixed": FSIM_MIXED}[prec_name]
    gb, D, Jo, Ko = spd3
    tol = 1e-10 if prec == FSIM_FP64 else 2e-6 * np.abs(Jo).max()
    gb.fock_build(D, tau=0.0, precision=prec)  # plan
    covered = {}
    for ps, cs in itertools.product((1, 3, 9, 27), (1, 2, 4)):
        code = 10 * ps + cs
        took = []
        for xy in PAIRS:
            try:
                gb.set_launch({xy: code}, tau=0.0, precision=prec)
                took.append(xy)
            except FsimError:
                gb.set_launch({xy: 11}, tau=0.0, precision=prec)  # shape not legal for this class pair
        J, K = gb.fock_build(D, tau=0.0, precision=prec)
        ej, ek = np.abs(J - Jo).max(), np.abs(K - Ko).max()
        assert ej < tol and ek < tol, (ps, cs, ej, ek)
        covered[code] = took
    # the cooperative kernel on every class pair
    gb.set_launch({xy: -1 for xy in PAIRS}, tau=0.0, precision=prec)
    J, K = gb.fock_build(D, tau=0.0, precision=prec)
    assert np.abs(J - Jo).max() < tol and np.abs(K - Ko).max() < tol
    # every shape reached the heaviest class pair, where the bench's tuned shapes live
    assert all((5, 5) in covered[10 * ps + cs] for ps in (1, 3, 9, 27) for cs in (1, 2, 4))
    assert len(covered[11]) == len(PAIRS)


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_split_shapes_ragged_primitive_counts(prec_name):
    from oracle import OracleBasis
    from paper_2510_24968_gb300 import FSIM_FP64, FSIM_MIXED, Basis, FsimError
    from .helpers import make_mol
    prec = {"fp64": FSIM_FP64, "mixed": FSIM_MIXED}[prec_name]
    rng = np.random.default_rng(2027)
    atoms, shells = [], []
    for a in range(3):
        atoms.append((int(rng.integers(1, 9)), tuple(rng.uniform(-1.6, 1.6, 3))))
        for l in range(3):
            for k in (1 + (a + l) % 4, 4 - (a + 2 * l) % 4):  # 1..4 primitives
                al = tuple(sorted(rng.uniform(0.2, 2.5, k)))
                shells.append((a, l, al, tuple(rng.uniform(0.2, 1.0, k))))
    mol = make_mol(atoms, shells, "ragged")
    gb, ob = Basis(mol), OracleBasis(mol)
    D = np.random.default_rng(79).standard_normal((gb.nbf, gb.nbf))
    D = D + D.T
    Jo, Ko, _ = ob.jk(D)
    tol = 1e-10 if prec == FSIM_FP64 else 2e-6 * np.abs(Jo).max()
    gb.fock_build(D, tau=0.0, precision=prec)
    for ps, cs in itertools.product((3, 9, 27), (1, 2, 4)):
        for xy in PAIRS:
            try:
                gb.set_launch({xy: 10 * ps + cs}, tau=0.0, precision=prec)
            except FsimError:  # fewer ket chunks than groups: the same split, one group
                gb.set_launch({xy: 10 * ps + 1}, tau=0.0, precision=prec)
        J, K = gb.fock_build(D, tau=0.0, precision=prec)
        ej, ek = np.abs(J - Jo).max(), np.abs(K - Ko).max()
        assert ej < tol and ek < tol, (ps, cs, ej, ek)


def test_hot_kernel_blocks_full_size_organic_cloud():
    # 60 heavy atoms, 1140 functions, tau 1e-11, mixed precision through the hot kernel;
    # D lives on the shells of three neighbouring atoms
    from oracle import OracleBasis
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis
    mol = workload("cloud60")
    gb, ob = Basis(mol), OracleBasis(mol)
    ls = [s.l for s in mol.shells]
    ao = np.cumsum([0] + [(l + 1) * (l + 2) // 2 for l in ls])
    atom_of = np.array([s.atom for s in mol.shells])
    xyz = np.asarray(mol.xyz)
    a0 = 17
    near = np.argsort(np.linalg.norm(xyz - xyz[a0], axis=1))[:3]
    sup = np.concatenate([np.arange(ao[i], ao[i + 1]) for i in range(mol.nshell) if atom_of[i] in near])
    rng = np.random.default_rng(60)
    D = np.zeros((gb.nbf, gb.nbf))
    blk = rng.standard_normal((sup.size, sup.size)) * 0.1
    D[np.ix_(sup, sup)] = blk + blk.T
    Q = ob.schwarz()
    Dt = torch.from_numpy(D).cuda()
    J, K = gb.fock_build(Dt, tau=1e-11, precision=FSIM_MIXED)
    J, K = J.cpu().numpy(), K.cpu().numpy()
    scale = np.abs(J).max()
    d_near = [i for i in range(mol.nshell) if atom_of[i] in near and ls[i] == 2]
    p_near = [i for i in range(mol.nshell) if atom_of[i] in near and ls[i] == 1]
    s_far = [i for i in range(mol.nshell) if atom_of[i] not in near and ls[i] == 0]
    for sa, sb in [(d_near[0], d_near[-1]), (d_near[1], p_near[2]), (p_near[0], s_far[5]), (d_near[0], s_far[40])]:
        Jb, Kb = ob.jk_block(D, sa, sb, tau=1e-11, Q=Q)
        sl = (slice(ao[sa], ao[sa + 1]), slice(ao[sb], ao[sb + 1]))
        assert np.abs(J[sl] - Jb).max() < 2e-6 * scale and np.abs(K[sl] - Kb).max() < 2e-6 * scale, (sa, sb)
