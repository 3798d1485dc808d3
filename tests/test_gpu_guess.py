"""Learned initial density: network kernels against the FP64 oracle network,
pair-local frames against rotation covariance, the guess check/fallback, and a
small end-to-end gain (fewer SCF iterations, same energy)."""
import math

import numpy as np
import pytest

from fsim_synth import water_cluster

from .helpers import make_mol

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_24968_gb300.build import build
    build()


def _net_and_data(width=32, b=300, seed=0):
    from paper_2510_24968_gb300.guess import GuessNet
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((b, 48)).astype(np.float32)
    t = rng.standard_normal((b, 225)).astype(np.float32) * 0.3
    m = (rng.random((b, 225)) > 0.5).astype(np.float32)
    net = GuessNet(width=width, seed=5)
    return net, x, t, m


def test_mlp_forward_and_gradient_match_fp64_oracle():
    from oracle import mlp
    net, x, t, m = _net_and_data()
    p = net.params().astype(np.float64)
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    y = torch.empty((x.shape[0], 225), dtype=torch.float32, device="cuda")
    yo, _ = mlp.forward(p, x.astype(np.float64), 48, 32, 225)
    net.forward(xd.data_ptr(), y.data_ptr(), x.shape[0], bf16=False)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - yo).max() < 1e-5 * max(1.0, np.abs(yo).max())
    net.forward(xd.data_ptr(), y.data_ptr(), x.shape[0], bf16=True)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - yo).max() < 3e-2 * max(1.0, np.abs(yo).max())
    loss, g = net.grad(xd.data_ptr(), td.data_ptr(), md.data_ptr(), x.shape[0], bf16=False)
    go = mlp.grad(p, x.astype(np.float64), t.astype(np.float64), m.astype(np.float64), 48, 32, 225)
    assert loss == pytest.approx(mlp.loss(p, x, t, m, 48, 32, 225), rel=1e-5)
    assert np.linalg.norm(g - go) / np.linalg.norm(go) < 1e-4
    _, gb = net.grad(xd.data_ptr(), td.data_ptr(), md.data_ptr(), x.shape[0], bf16=True)
    assert np.linalg.norm(gb - go) / np.linalg.norm(go) < 5e-2


def _bf16(a):
    """Round FP32 values to BF16 (round to nearest even), kept as FP32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("width", [32, 256])
def test_mlp_bf16_forward_is_the_bf16_operand_product(width):
    # the BF16 forward pass is the network with every GEMM operand rounded to
    # BF16 and products accumulated in FP32 (tensor cores): against that
    # definition in FP64 it agrees to accumulation order and rare one-ulp BF16
    # differences of the FP32-computed activations; batch 300 spans three
    # 128-row tiles, width 256 four 64-wide K chunks, 225 outputs two column tiles
    net, x, t, m = _net_and_data(width=width)
    p = net.params().astype(np.float32)
    nin, nout, w = 48, 225, width
    sizes = [nin * w, w, w * w, w, w * nout, nout]
    parts = np.split(p, np.cumsum(sizes)[:-1])
    W1, b1, W2, b2, W3, b3 = (parts[0].reshape(nin, w), parts[1], parts[2].reshape(w, w), parts[3],
                              parts[4].reshape(w, nout), parts[5])

    def lin(h, W, b):
        return _bf16(h).astype(np.float64) @ _bf16(W).astype(np.float64) + b

    def silu(z):
        return z / (1.0 + np.exp(-z))

    h1 = silu(lin(x, W1, b1)).astype(np.float32)
    h2 = silu(lin(h1, W2, b2)).astype(np.float32)
    yref = lin(h2, W3, b3)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((x.shape[0], nout), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), y.data_ptr(), x.shape[0], bf16=True)
    torch.cuda.synchronize()
    assert np.abs(y.cpu().numpy() - yref).max() < 2e-3 * np.abs(yref).max()


def test_training_reduces_loss():
    from paper_2510_24968_gb300.guess import train
    net, x, t, m = _net_and_data(width=64, b=512, seed=1)
    losses = train(net, x, t * 0 + np.tanh(x[:, :1]) * 0.5, m, steps=200, batch=256, lr0=3e-3, log_every=50)
    assert losses[-1][1] < 0.25 * losses[0][1]


def _rotated(mol, th=0.9):
    Rm = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    Rm = Rm @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)], [0, math.sin(0.4), math.cos(0.4)]])
    return make_mol([(z, tuple(Rm @ x + np.array([0.3, -1.1, 2.0]))) for z, x in zip(mol.Z, mol.xyz)],
                    [(s.atom, s.l, s.alpha, s.coef) for s in mol.shells])


def test_local_blocks_rotation_invariant_and_round_trip():
    from paper_2510_24968_gb300 import FSIM_FP64, Basis
    from paper_2510_24968_gb300.guess import features, load, targets, _check
    import ctypes as C
    mol = water_cluster(2, geom_seed=21)
    b1, b2 = Basis(mol), Basis(_rotated(mol))
    r1 = b1.scf(precision=FSIM_FP64, tau=1e-12, want_density=True)
    r2 = b2.scf(precision=FSIM_FP64, tau=1e-12, want_density=True)
    assert abs(r1["e_total"] - r2["e_total"]) < 1e-9
    assert np.abs(features(b1) - features(b2)).max() < 1e-5
    t1, m1 = targets(b1, r1["D"])
    t2, m2 = targets(b2, r2["D"])
    assert np.array_equal(m1, m2)
    assert np.abs(t1 - t2).max() < 1e-5
    # assembling the exact local blocks gives back the density
    y = torch.from_numpy(t1).cuda()
    D = torch.zeros((b1.nbf, b1.nbf), dtype=torch.float64, device="cuda")
    _check(load().fsim_guess_assemble(b1.h, C.c_void_p(y.data_ptr()), C.c_void_p(D.data_ptr()), None))
    assert np.abs(D.cpu().numpy() - r1["D"]).max() < 1e-5 * max(1.0, np.abs(r1["D"]).max())


def test_bad_guess_falls_back_to_core():
    from paper_2510_24968_gb300 import FSIM_FP64, Basis
    b = Basis(water_cluster(2, geom_seed=3))
    core = b.scf(precision=FSIM_FP64, tau=1e-10)
    bad = b.scf(precision=FSIM_FP64, tau=1e-10, D0=np.zeros((b.nbf, b.nbf)))
    assert bad["guess_fallback"] and bad["iters"] == core["iters"]
    assert abs(bad["e_total"] - core["e_total"]) < 1e-10


def test_learned_guess_saves_iterations_small(tmp_path):
    # the network's guess, supplied as D0 and run inside fsim_scf from its weights
    # file (FSIM_GUESS_LEARNED): fewer iterations than core-H, the same energy
    from paper_2510_24968_gb300 import FSIM_MIXED, Basis
    from paper_2510_24968_gb300.guess import GuessNet, predict_density, train, training_data
    train_mols = [water_cluster(k, geom_seed=10**6 + i) for i, k in enumerate([2, 3, 4] * 20)]
    X, T, M, _ = training_data(train_mols)
    net = GuessNet(seed=3)
    train(net, X, T, M, steps=1500, batch=2048, lr0=1e-3)
    path = tmp_path / "guess.fsimmlp"
    net.save(path)
    gain = []
    for i in range(2):
        b = Basis(water_cluster(4, geom_seed=2 * 10**6 + i))
        core = b.scf(precision=FSIM_MIXED, tau=1e-10)
        learned = b.scf(precision=FSIM_MIXED, tau=1e-10, D0=predict_density(b, net))
        inlib = b.scf(precision=FSIM_MIXED, tau=1e-10, guess_model=path)
        assert core["converged"] and learned["converged"] and not learned["guess_fallback"]
        assert abs(learned["e_total"] - core["e_total"]) < 1e-8
        assert inlib["converged"] and not inlib["guess_fallback"] and inlib["guess_s"] > 0
        assert abs(inlib["e_total"] - core["e_total"]) < 1e-8 and abs(inlib["iters"] - learned["iters"]) <= 1
        gain.append(core["iters"] - learned["iters"])
    assert sum(gain) > 0


def test_weights_file_round_trip_and_rejections(tmp_path):
    from paper_2510_24968_gb300 import FSIM_FP64, Basis, FsimError
    from paper_2510_24968_gb300.fsim import load
    from paper_2510_24968_gb300.guess import GuessNet
    import ctypes as C
    import os
    net = GuessNet(width=40, seed=9)
    path = tmp_path / "w.fsimmlp"
    net.save(path)
    h = C.c_void_p()
    assert load().fsim_mlp_load(os.fsencode(path), C.byref(h)) == 0
    back = GuessNet.__new__(GuessNet)
    back.h, back.np = h, load().fsim_mlp_nparams(h)
    assert np.array_equal(back.params(), net.params())
    b = Basis(water_cluster(2, geom_seed=3))
    # a network whose output width is not the block layout's
    bad = GuessNet(nout=100, seed=1)
    bad.save(tmp_path / "bad.fsimmlp")
    with pytest.raises(FsimError):
        b.scf(precision=FSIM_FP64, tau=1e-10, guess_model=tmp_path / "bad.fsimmlp")
    # a file that is not a weights file
    (tmp_path / "junk").write_bytes(b"FSIMMLP1" + b"\x00" * 7)
    with pytest.raises(FsimError):
        b.scf(precision=FSIM_FP64, tau=1e-10, guess_model=tmp_path / "junk")


@pytest.mark.parametrize("k,seed", [(2, 6), (4, 8)])
def test_frames_features_blocks_match_oracle(k, seed):
    # the library's pair features, local blocks and assembly against the numpy
    # restatement (oracle/guess.py, whose rotation matrices come from least squares)
    import ctypes as C
    from oracle import OracleBasis
    from oracle import guess as og
    from paper_2510_24968_gb300 import Basis
    from paper_2510_24968_gb300.guess import _check, features, load, targets
    mol = water_cluster(k, geom_seed=seed)
    b = Basis(mol)
    assert np.abs(features(b) - og.features(mol)).max() < 1e-6
    D = np.linalg.inv(OracleBasis(mol).onee("S"))
    t, m = targets(b, D)
    to, mo = og.targets(mol, D)
    assert np.array_equal(m, mo.astype(np.float32))
    assert np.abs(t - to).max() < 1e-6 * np.abs(to).max()
    # assembly of the same float32 blocks
    y = torch.from_numpy(t).cuda()
    Dg = torch.zeros((b.nbf, b.nbf), dtype=torch.float64, device="cuda")
    _check(load().fsim_guess_assemble(b.h, C.c_void_p(y.data_ptr()), C.c_void_p(Dg.data_ptr()), None))
    Do = og.assemble(mol, t.astype(np.float64))
    assert np.abs(Dg.cpu().numpy() - Do).max() < 1e-10 * max(1.0, np.abs(Do).max())


def test_adam_step_from_combined_shares_equals_train_step():
    # data-parallel update on one device, its two halves checked sharply:
    # (1) the gradients of two shares of a minibatch, weighted by their mask sums,
    #     are the whole minibatch's gradient (FP32 GEMMs: to rounding);
    # (2) fsim_mlp_adam_step fed the whole minibatch's gradient takes the same step
    #     as fsim_mlp_train_step (same BF16 kernels, same gradient)
    from paper_2510_24968_gb300.guess import GuessNet
    net, x, t, m = _net_and_data(width=64, b=512, seed=4)
    twin = GuessNet(width=64, seed=5)
    assert np.array_equal(twin.params(), net.params())
    xd, td, md = (torch.from_numpy(a).cuda() for a in (x, t, m))
    _, gfull = net.grad(xd.data_ptr(), td.data_ptr(), md.data_ptr(), 512, bf16=False)
    num, den = 0.0, 0.0
    for sl in (slice(0, 200), slice(200, 512)):
        xs, ts, ms = xd[sl].contiguous(), td[sl].contiguous(), md[sl].contiguous()
        _, g = net.grad(xs.data_ptr(), ts.data_ptr(), ms.data_ptr(), ms.shape[0], bf16=False)
        w = float(ms.sum().item())
        num, den = num + g.astype(np.float64) * w, den + w
    assert np.linalg.norm(num / den - gfull) < 1e-5 * np.linalg.norm(gfull)
    for step in range(3):
        _, g = twin.grad(xd.data_ptr(), td.data_ptr(), md.data_ptr(), 512, bf16=True)
        twin.adam_step(g, 1e-3)
        net.train_step(xd.data_ptr(), td.data_ptr(), md.data_ptr(), 512, 1e-3)
        torch.cuda.synchronize()
    pa, pb = net.params(), twin.params()
    assert np.abs(pa - pb).max() <= 1e-6 * max(1.0, np.abs(pa).max())
